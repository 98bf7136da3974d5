// Host-side setup of the space-time FE hierarchy (arXiv 2303.06742, Secs. 2-4).
// Builds, per multigrid level, the spatial system matrix whose Kronecker
// combination with the temporal matrices gives the slab matrix of Problem 4.1,
// plus transfers, vertex patches, patch inverses and the coarse inverse.
#pragma once
#include <cstdint>
#include <memory>
#include <new>
#include <type_traits>
#include <string>
#include <utility>
#include <vector>

#include "../../include/stfem.h"

namespace stfem {

// Allocator whose value-less construct leaves the element uninitialised, so
// that resize() of a large array costs no serial write: the threaded loop that
// fills it touches its pages first.
template <class T> struct uninit_alloc : std::allocator<T> {
  template <class U> struct rebind {
    using other = uninit_alloc<U>;
  };
  uninit_alloc() = default;
  template <class U> uninit_alloc(const uninit_alloc<U> &) noexcept {}
  template <class U> void construct(U *p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new ((void *)p) U;
  }
  template <class U, class... A> void construct(U *p, A &&...a) { ::new ((void *)p) U(std::forward<A>(a)...); }
};
template <class T> using hvec = std::vector<T, uninit_alloc<T>>;

struct Rule {
  std::vector<double> x, w;
};

Rule gauss01(int n);                  // n-point Gauss-Legendre on [0,1]
std::vector<double> lobatto01(int r); // r+1 Gauss-Lobatto points on [0,1]
Rule radau_right(int n);              // n-point right Gauss-Radau on [-1,1] (Eq. 2.4)
// Lagrange basis on `nodes` at x: values val[i], derivatives der[i].
void lagrange(const std::vector<double> &nodes, double x, double *val, double *der);

// dG(k) temporal data: Radau nodes/weights on [-1,1], chi_a(-1) and
// Dt[b*q+a] = w_b chi_a'(t_b) + chi_a(-1) chi_b(-1).
struct Temporal {
  int k = 0, q = 1;
  std::vector<double> t, w, chi_m1, Dt;
};
Temporal make_temporal(int k);

struct Box {
  int dim = 2;
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  double vol = 1, hF = 1;
  long ncell = 1;
};
Box make_box(int dim, const double *lo, const double *hi, const int *n, int hf_mode);

struct Coef {
  double rho = 1, alpha = 1, c0 = 1;
  std::vector<double> lam, mu, kap; // per cell of the level
  // permeability tensor per cell (dim x dim, row-major); empty: K = kap I
  std::vector<double> K;
};
Coef coarsen(const Coef &fine, const Box &fine_box);

struct BCs {
  int bc_u[6] = {0, 0, 0, 0, 0, 0};
  int bc_p[6] = {0, 0, 0, 0, 0, 0};
};

// A scalar Lagrange lattice space Q_m on a box.
struct Lattice {
  int dim = 2, m = 1;
  int dims[3] = {1, 1, 1};
  long nnodes = 1;
  std::vector<double> ref; // Gauss-Lobatto points on [0,1]
};
Lattice make_lattice(const Box &b, int m);
// Range of cells (along one axis) whose closure holds lattice coordinate a.
void cells_of(int a, int m, int ncell, int *c_lo, int *c_hi);

// Spatial system matrix of one level: rows (u-eq, v-eq, p-eq), columns
// (V, U, P); entry (v1, v2) multiplies Dt and W respectively, so that
// (A x)_b = sum_a Dt[b,a] S1 x_a + W_b S2 x_b.
struct Level {
  Box box;
  int r = 2;
  Lattice U, P;
  long R = 0, S = 0, ns = 0;
  Coef coef;
  std::vector<int> rowptr;
  hvec<int> col;
  hvec<double> v1, v2;
  // STFEM_FORM_PROBLEM_3_1: the p-equation couples -C to V (in v2);
  // STFEM_FORM_PROBLEM_B_1: to U (in v1).  For B.1 an assembled level also
  // keeps -Cvol, the volume part of the same coupling, per pressure node over
  // its displacement neighbour box (d values per neighbour, the order of the
  // p-rows' entries): the previous-slab coupling of Problem B.1 uses it.
  int form = 0;
  std::vector<double> cvol;
  // STFEM_PRESSURE_BROKEN: P is P_{r-1}^disc, numbered cell by cell (cells x
  // fastest, pnloc dofs each: Legendre products of total degree <= r-1, x
  // exponent fastest); P.nnodes counts its dofs and P.dims is unused.
  bool pdisc = false;
  int pnloc = 0;
  // Unit-coefficient element matrices of the level's cells (uniform mesh, so
  // one set serves every cell), kept for the matrix-free operator (continuous
  // pressure only).  Row-major; u dofs i * d + c (i < nu local Q_r nodes),
  // p dofs s (np local Q_{r-1} nodes); local nodes lexicographic, x fastest,
  // with lattice offsets locu / locp (3 per node).  A cell with lambda, mu,
  // kappa has K = lam Klam + mu Kmu (+ per Dirichlet-u face f:
  // lam fKlam[f] + mu fKmu[f] + fKpen[f]), C = Cv (+ fC[f]), the mass rho Mu
  // (per component) and c0 Mp, B = kap Bv (+ per Dirichlet-p face:
  // kap fB[f] + fBpen[f]); f = 2 axis + side.  alpha is part of Cv and fC.
  struct Elem {
    int nu = 0, np = 0;
    std::vector<int> locu, locp;
    std::vector<double> Mu, Kmu, Klam, Cv, Bv, Mp;
    std::vector<double> fKmu[6], fKlam[6], fKpen[6], fC[6], fB[6], fBpen[6];
  } elem;
  BCs bc;
};

Level assemble_level(const Box &b, int r, const Coef &c, const BCs &bc, int form = 0, int pressure = 0);

// Basis data of a level's two spaces at the quadrature points of each face
// f = 2 * axis + side of a cell (Gauss-Legendre with r + 2 points per
// direction, as for the matrices), for the boundary data terms of Eq. 3.4.
// Arrays are face-major: reference points x [f][pt][3], weights w [f][pt]
// (the face measure included), displacement values U [f][pt][nu] and
// physical gradients dU [f][pt][nu][d], and the same (P, dP, np local
// functions) for the pressure space, broken or continuous.  Local functions
// are numbered as in the cell loads.
struct FaceTables {
  int npts = 0, nu = 0, np = 0;
  std::vector<double> x, w, U, dU, P, dP;
};
void face_tables(const Level &L, FaceTables *out);
// Embedding of the broken P_m space of the coarse box into that of the fine
// box (nested; fine rows, coarse columns).
struct CSR;
CSR prolongation_disc(int m, const Box &cb, const Box &fb);

// Scalar interpolation coarse Q_m -> fine Q_m (fine rows), CSR.
struct CSR {
  long nrows = 0, ncols = 0;
  std::vector<int> rowptr, col;
  std::vector<double> val;
};
CSR prolongation(const Lattice &coarse, const Box &cbox, const Lattice &fine, const Box &fbox);
CSR transpose(const CSR &a);
// Galerkin product P_s^T S P_s of the spatial system of `fine` (both value
// arrays), P_s = blockdiag(Pu (x) I_d, Pu (x) I_d, Pp); fills the matrix of
// `coarse` (whose sizes must be set).  Works on the node-level blocks of the
// system; false if `fine` does not have that block structure.
bool galerkin(const Level &fine, const CSR &Pu, const CSR &Pp, Level *coarse);

// Eigen-decomposition of W^{-1} Dt = V diag(lam) V^{-1} used by the
// time-diagonal form of the patch inverses.  Slots: the nr real eigenvalues
// first, then one member (Im > 0) of each of the nc complex-conjugate pairs.
// U = V^{-1} W^{-1}; rows/columns are given for the slots only (the partner of
// a pair is the complex conjugate).  All arrays row-major, complex as (re, im).
struct TimeDiag {
  int q = 0, nr = 0, nc = 0;
  std::vector<double> lam;  // [slot][2]
  std::vector<double> Vmat; // [b][slot][2]: V[b][a]
  std::vector<double> Umat; // [slot][b][2]: U[a][b]
};
// Fails (returns false) when W^{-1} Dt is not diagonalisable to 1e-10.
bool time_diag(const Temporal &T, double tau, TimeDiag *out, std::string *err);

// Vertex patches of a level (reading: dofs whose support lies in the closed
// patch), with the patch matrices inverted in FP64.
//
// form 0 (dense): per patch the column-major C x C inverse, leading dim ld.
// form 1 (time-diagonal): per patch, for each real slot the column-major
// (lam S1_P + S2_P)^{-1} (Cs x Cs, leading dim ldR = ceil(Cs/4)*4), then for each
// complex slot the same for complex lam with (re, im) interleaved per row
// (leading dim ldC = 2*ceil(Cs/2)*2 reals).
struct Patches {
  long npatch = 0;
  std::vector<int> size;          // C_P
  std::vector<long long> dof_off; // offset into dofs
  std::vector<int> dofs;          // global slab indices (paper order)
  std::vector<long long> inv_off; // offset (elements) into inv
  std::vector<double> inv;        // column-major A_P^{-1}, leading dim ld(C_P)
  std::vector<int> ld;
  int form = 0;
  std::vector<int> cs;            // spatial size Cs of each patch (form 1)
};
// vec: elements per 16-byte vector of the storage type (2 for FP64, 4 for FP32).
// invert_them = false only builds the dof lists.  td != nullptr selects the
// time-diagonal form.  kind 0: vertex patches (Eq. 4.9, nodes supported in
// the closed patch); kind 1: cell patches (every node of the closed cell).
int build_patches(const Level &L, const Temporal &T, double tau, int vec, Patches *out,
                  std::string *err, bool invert_them = true, const TimeDiag *td = nullptr, int kind = 0);

// The spatial patch blocks S1_P, S2_P (row-major C_s x C_s each, S2 right
// after S1) of patches p0 .. p1-1 of a level whose dof lists P holds (built
// with invert_them = false), for inversion on the device; off[p - p0] is
// the offset of patch p's S1 in out.  Threaded.
void extract_patch_blocks(const Level &L, const Patches &P, int q, long p0, long p1, hvec<double> *out,
                          std::vector<long long> *off);

// Values of the broken P_m basis (Legendre products of total degree <= m,
// x exponent fastest) at npts reference points xi[3 * i + axis] of the unit
// cell: phi[i * nloc + l].  Returns nloc.
int disc_basis(int m, int dim, const double *xi, int npts, std::vector<double> *phi);

// y = A_n x of a level (q time nodes; Dt and W of Eq. 4.7) computed on the
// host from the node-block arrays the device operator reads (defined with the
// kernels): a CPU check of that layout.  x, y: host, q * ns.
int block_apply_level(const Level &L, int q, const double *Dt, const double *W, const double *x, double *y,
                      std::string *err);

// Dense row-major slab matrix of a level (for the coarse solve).
std::vector<double> dense_slab(const Level &L, const Temporal &T, double tau);
// In-place Gauss-Jordan inverse with partial pivoting of a row-major n x n
// matrix. Returns false on a zero pivot.
bool invert(double *a, int n);

int n_threads();

// Validates the ABI arguments and builds every level (finest last) and the
// scalar transfers Pu[l], Pp[l] from level l-1 to l (index 0 unused).
int build_hierarchy(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                    const stfem_bcs *bcs, double tau, std::vector<Level> *levels, std::vector<CSR> *Pu,
                    std::vector<CSR> *Pp, std::string *err);

} // namespace stfem
