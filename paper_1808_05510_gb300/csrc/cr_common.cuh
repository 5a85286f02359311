// Internal declarations shared by the CUDA translation units of libconreg.
//
// Device data layout (all float64 unless noted, column-major):
//   UU (ny x 3 r_cap): column 3p+s holds L_y^s u_p (s = 0, 1, 2); VV likewise
//   for v_p and L_x.  Interleaving puts every factor block that the residual
//   products and the residual norm need (Sec. 2.3: R_j v, R_j^T u) into one
//   contiguous panel, so each of them is a single panel-times-vector pass.
//   E (ny x m) = Omega o (Y - U Z V^T X): the masked data residual, refreshed
//   once per projection; R_j v = E (X^T v) - UU g(v) with a 3j coefficient
//   vector g (see cr_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include <atomic>

#include <string>
#include <vector>

#include "conreg.h"

struct cr_net;

namespace cr {

// Host copies of a descriptor's device arrays (cr_problem_desc.mem_kind = CR_MEM_DEVICE).
struct DescCopy {
  std::vector<int32_t> lx_rp, lx_col, ly_rp, ly_col, gx, gy;
  std::vector<double> lx_val, ly_val, X, Y;
  std::vector<uint8_t> Om;
};
// Stage a device descriptor into *store (host view in *view); host descriptors pass through.
cr_status stage_desc(const cr_problem_desc* d, DescCopy* store, cr_problem_desc* view, std::string& err);
}  // namespace cr

namespace cr {

// Number of kernels this library has launched (process-wide).
extern std::atomic<long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kMaxSlots = 16;     // off-diagonal entries per Laplacian row
constexpr int kPcgThreads = 512;  // threads per CTA of the cluster PCG
constexpr int kMaxCluster = 16;

// Sparse symmetric matrix in padded ELL form ("slot-major": slot k of row i at
// [k * n + i]); the diagonal is kept apart.  Graph Laplacians with unit weights
// store no off-diagonal values (offw == nullptr; every stored neighbour has
// weight -1).  For the cluster PCG the neighbour of slot k is also stored
// packed as (cta_rank << 24) | local_index for the partition of the rows into
// contiguous chunks of `chunk` rows, one chunk per CTA of a cluster of `csize`.
struct DevLap {
  int n = 0;
  int K = 0;                     // slots per row (padded entries are -1)
  const int* nbr = nullptr;      // [K * n] global column, -1 = none
  const int* nbrp = nullptr;     // [K * n] packed (rank, local), -1 = none
  const double* offw = nullptr;  // [K * n] or nullptr (unit Laplacian)
  const double* diag = nullptr;  // [n]  L_ii
  const double* l2diag = nullptr;// [n]  (L^2)_ii = L_ii^2 + sum_k L_ik^2
  int chunk = 0;                 // rows per CTA
  int csize = 1;                 // CTAs per cluster
};

// X restricted to the rows owned by each CTA of the PCG partition (v side):
// for CTA r and injection a, entries lx_ptr[r*m + a] .. lx_ptr[r*m + a + 1] - 1
// hold (local row, value).  Plus the CSR of X by row (global rows).
struct DevXLocal {
  const int* lx_ptr = nullptr;
  const int* lx_row = nullptr;
  const double* lx_val = nullptr;
  const int* xr_ptr = nullptr;   // [nx + 1]
  const int* xr_col = nullptr;
  const double* xr_val = nullptr;
  const float* lx_valf = nullptr;  // float32 copies (mixed form)
  const float* xr_valf = nullptr;
};

// Scalars the host reads back after a PCG solve.
struct PcgStat {
  int iters;
  int status;      // 0 ok, 1 hit maxit, 2 breakdown
  double relres;   // recursive residual estimate at exit
  double bnorm;
};

// One PCG solve with the operator  lam * [(L + c I)^2 + e I] + data,  where
// c = coef[0], e = coef[1] - coef[0]^2 (both read on the device), and
//   data = diag(omega_tilde),  omega_tilde_i = sum_a Om[i + a ldo] * xi[a]^2   (u side, Eq. ALS_linsys)
//   data = X diag(s) X^T                                                        (v side, Eq. ALS_linsys_v)
struct PcgArgs {
  DevLap L;
  double lam;
  const double* coef;      // device [2]: (c, d)
  int m;
  const uint8_t* Om;       // u side
  int64_t ldo;
  const double* xi;        // u side: device [m]
  DevXLocal X;             // v side
  const double* s;         // v side: device [m]
  const double* b;         // rhs [n]
  double* x;               // in: x0, out: solution [n]
  double* r;               // work [n]
  double* p;               // work [n]
  double* sv;              // work [n]
  double* w;               // work [n]
  double* dinv;            // work [n]
  double* omt;             // work [n] (u side)
  double tol;
  int maxit;
  PcgStat* stat;           // device
  int force_generic;       // 1: always use the shared/global-memory kernel
  int fp32;                // 1: float32 vectors and arithmetic, float64 inner products and scalars
};

// ---------------------------------------------------------------- cr_mg.cu
// Multigrid preconditioner of the ALS sub-problems: the hierarchy of one
// Laplacian (built on the host by cr_mg_host.h) in device memory.  Level 0 is
// the fine grid itself (DevLap, partitioned in chunks of L.chunk rows over the
// cluster); levels l >= 1 keep L_l and M_l entry by entry so that the kernel
// forms L_l + sigma M_l for any shift.  Column references are packed as
// (owner CTA << 24) | local row in the owner's partition of the referenced level.
constexpr int kMgMaxLev = 8;
constexpr int kMgCoarseMax = 64;  // rows of the coarsest level (solved through its eigenbasis)
constexpr int kMgTailRows = 512;  // levels of at most this many rows run on CTA 0 alone

struct DevMgLevel {
  int n = 0;       // rows
  int chunk = 0;   // rows per CTA when distributed; n when on CTA 0 alone
  int dist = 0;    // 1: distributed over the cluster, 0: CTA 0 alone
  int off = 0;     // offset of the level's five work vectors in the kernel's shared memory (elements)
  // operator rows (levels >= 1): CSR by global row, packed column refs, values of L_l and M_l
  const int* rp = nullptr;
  const int* cp = nullptr;
  const double* lv = nullptr;
  const double* mv = nullptr;
  const double* dl = nullptr;  // diagonals of L_l and M_l
  const double* dm = nullptr;
  // prolongation from level l+1 (CSR by row of this level, refs into level l+1)
  const int* prp = nullptr;
  const int* pcp = nullptr;
  const double* pv = nullptr;
  // restriction into level l+1 (CSR by row of level l+1, refs into this level)
  const int* rrp = nullptr;
  const int* rcp = nullptr;
  const double* rv = nullptr;
  // This level's sections of a CTA's tables (byte offsets from the CTA's table
  // base): operator rows (levels 1 .. nlev-2), prolongation rows (level l's own
  // rows), restriction rows (level l+1's own rows).  Each section: a local row
  // pointer (rows + 1 ints), then the entries' 32-bit cluster addresses, then
  // their coefficients (8-byte slots).
  int64_t op_rp = 0, op_a = 0, op_c = 0;
  int64_t p_rp = 0, p_a = 0, p_c = 0;
  int64_t r_rp = 0, r_a = 0, r_c = 0;
};

struct DevMg {
  int nlev = 0;                // levels, the last one the coarsest (CTA 0, dense)
  int ld = 0;                  // first level that runs on CTA 0 alone
  int nc = 0;                  // rows of the coarsest level
  DevMgLevel lev[kMgMaxLev];
  // (L_c + sigma M_c)^-1 = Q diag(1 / (mu + sigma)) Q^T on the coarsest level
  const double* cQ = nullptr;  // nc x nc, column-major
  const double* cmu = nullptr; // nc
  const double* xn2 = nullptr; // v side: |X_a|^2 per injection (mean data weight of the shift)
  int lvl_elems = 0;           // shared-memory elements of the levels >= 1
  // algorithmic bytes of one PCG iteration ([0] float32, [1] float64; host accounting):
  // the fine-level PCG as the Jacobi count plus, for each of the two V-cycles, four
  // sweeps, restriction and prolongation per level and the coarsest dense solve
  double bytes_iter[2] = {0.0, 0.0};
  size_t smem[2] = {0, 0};     // dynamic shared memory of the kernel for T = float, double (0: does not fit)
  // Tables each CTA fills at launch for the rows it owns: the 32-bit
  // cluster-window address of every referenced entry (relative to its level's
  // first vector) and its coefficient in the solve's precision.  Level 0's
  // neighbour addresses (slot-major, K x chunk0; a missing neighbour points at a
  // zero word) and coefficients (weighted Laplacians only) and its diagonal come
  // first, then each level's sections.  They live in the CTA's shared memory
  // when they fit (tab_smem), else in tab_glob + rank * tab_bytes.
  int64_t nb_a = 0, nb_c = -1, dg = 0;  // byte offsets; nb_c < 0: unit weights (coefficient -1)
  int64_t tab_bytes = 0;               // bytes of one CTA's tables
  int tab_smem[2] = {0, 0};            // tables in shared memory for T = float, double
  char* tab_glob = nullptr;            // csize * tab_bytes bytes when a precision keeps them in global memory
  // v side, ninj <= kMgSmwMax: Sherman-Morrison-Woodbury correction of the preconditioner for the
  // rank-ninj data term X diag(s) X^T.  Cached per problem: MX = M0^-1 X (n x ninj, row i at i * ninj,
  // in the kernel's precision), X^T MX (ninj x ninj, float64) and the shift they were formed with.
  int smw = 0;
  double* smw_mx = nullptr;
  double* smw_xx = nullptr;
  double* smw_sig = nullptr;  // [0]: the shift MX was formed with (0 = none), [1]: its precision (bytes of T)
};
constexpr int kMgSmwMax = 32;

// Dynamic shared memory of the multigrid PCG for T (bytes), from the level sizes,
// without (tables = false) or with the CTA's tables.
size_t mg_smem_bytes(const DevMg& g, int chunk0, int m, bool fp32, bool tables);
// Kernel attributes for the multigrid PCG (cluster size up to 16, large shared memory).
cudaError_t mg_prepare();
// Whether a cluster of csize CTAs with smem bytes each fits on this device (after mg_prepare).
bool mg_cluster_ok(int csize, size_t smem, bool fp32);
// One PCG solve of the system of `a` (side 0: Eq. ALS_linsys, 1: Eq. ALS_linsys_v)
// preconditioned by two V-cycles of L + sigma I (scaled by 1 / lam), on the cluster
// partition of a.L.  a.x is the initial guess and the result; a.p, a.sv, a.omt are work.
cudaError_t mg_pcg_launch(const PcgArgs& a, const DevMg& g, int side, cudaStream_t st);

// ---------------------------------------------------------------- cr_pcg_grid.cu
// Grid-wide PCG (vectors in HBM, all SMs) for grids the register-resident cluster kernel does not take.
// Blocks of the cooperative launch (0: cannot run) and work doubles needed.
int pcg_grid_blocks(bool fp32, int m, int K);
size_t pcg_grid_work_elems(int n);
// Solves the system of `a` (side 0: Eq. ALS_linsys, 1: Eq. ALS_linsys_v) with
// a.dinv, a.omt precomputed in float64 (fcg_jacobi_diag).  work: 9n doubles;
// part: nb*4, ypart: nb*m, yglob: m doubles; bar: 2 unsigned; err: 1 int.
// a.stat receives iterations and status (3 = grid barrier timed out).
cudaError_t pcg_grid_launch(const PcgArgs& a, int side, const int* xc_ptr, const int* xc_row, const double* xc_val,
                            double* work, double* part, double* ypart, double* yglob, unsigned* bar, int* err,
                            int nb, cudaStream_t st);

// ---------------------------------------------------------------- cr_pcg.cu
cudaError_t pcg_launch(const PcgArgs& a, int data_kind, cudaStream_t st);
cudaError_t pcg_prepare(int data_kind, int csize, size_t smem_bytes);
size_t pcg_smem_bytes(int chunk, int m);
// rows per thread of the register-resident cluster kernel for this operator, 0 if it does not apply
int pcg_reg_vpt(const DevLap& L, bool fp32);
bool pcg_cluster_ok(int csize, size_t smem_bytes);
// y = (L + shift I) x
void lap_apply(const DevLap& L, const double* x, double* y, double shift, cudaStream_t st);

// ---------------------------------------------------------------- cr_blas.cu
// Strided matrix view: element (i, k) at ptr[i * si + k * sk].
struct MatView {
  const double* ptr;
  int64_t si, sk;
};

// C(i, l) = alpha * sum_k A(i, k) B(k, l) + beta * C(i, l), for i < M, l < N,
// k < K.  Deterministic: K is split in a fixed number of ranges whose partial
// sums are added in order.  ws must hold splits * M * N doubles (see gemm_ws).
void gemm(int M, int N, int K, double alpha, MatView A, MatView B, double beta, double* C, int64_t sci,
          int64_t scl, double* ws, size_t ws_elems, cudaStream_t st);

// out[p * ostride] = alpha * sum_i A[i + p*lda] * w[i] (+ beta * out), p < k; one warp per column.
void gemv_t(int n, int k, const double* A, int64_t lda, const double* w, double* out, int64_t ostride,
            double alpha, double beta, cudaStream_t st);
// y[i] = beta * y[i] + alpha * sum_p A[i + p*lda] * c[p*cstride]
void gemv_n(int n, int k, const double* A, int64_t lda, const double* c, int64_t cstride, double* y,
            double alpha, double beta, cudaStream_t st);
// out = alpha * sum_i x[i] * y[i] into *out (single deterministic reduction)
void dot(int n, const double* x, const double* y, double* out, cudaStream_t st);
// out[a * ostride] = sum over the nonzeros of column a of X (CSC) of X_ka * v[k]
void spmv_xt(int m, const int* colptr, const int* row, const double* val, const double* v, double* out,
             int64_t ostride, cudaStream_t st);
// y[k] = beta*y[k] + alpha * sum_a X_ka * c[a], X by rows (CSR)
void spmv_x(int n, const int* rowptr, const int* col, const double* val, const double* c, double* y,
            double alpha, double beta, cudaStream_t st);
// out[a] = sum_i Om[i + a*ldo] * u[i]^2
void omega_sq_dots(int n, int m, const uint8_t* Om, int64_t ldo, const double* u, double* out,
                   cudaStream_t st);
// y = x * (1 / *nrm) ; *nrm computed on the device (sqrt of a dot)
void scale_by_inv_norm(int n, const double* x, const double* nrm2, double* y, cudaStream_t st);
void copy(int n, const double* x, double* y, cudaStream_t st);
void fill(int64_t n, double v, double* y, cudaStream_t st);

// Galerkin-specific kernels
// g_a = G_a w_a for a < m: G (m blocks of ld_g x ld_g, block a at G + a*gstride), w (j x m, ld ldw)
void batched_gemv(int j, int m, const double* G, int64_t ldg, int64_t gstride, const double* w, int64_t ldw,
                  double* out, int64_t ldo, cudaStream_t st);

// ---------------------------------------------------------------- cr_galerkin.cu
// CTAs of the persistent Galerkin CG (one per SM), 0 if the kernel cannot run.
int galerkin_grid_size();
// Eigenbasis form of the Galerkin CG: Qa (j x j, ld) the eigenvectors of A1,
// la, lb the eigenvalues of A1 and B1; Y, Gt ld x m work.  The launch's A2, B2,
// H, F, Z and Dg are then the transformed A2t, B2t, Ht, Ft, Zt and diagonal.
// With Ci set (m <= 128), the CG is preconditioned row by row by Sherman-Morrison-
// Woodbury (Dl, Hg, Ci from galerkin_eig_diag and galerkin_smw_setup, float64 in
// both instantiations; S ld x m and Yd j x j float64 work, Zz j x j work);
// otherwise by the diagonal Dg.
template <class T>
struct GalEig {
  const T *Qa = nullptr, *la = nullptr, *lb = nullptr;
  T *Y = nullptr, *Gt = nullptr;
  const double *Dl = nullptr, *Hg = nullptr, *Ci = nullptr;
  double *S = nullptr, *Yd = nullptr;
  T* Zz = nullptr;
};
// Arrowhead eigen-update of both eigenbases (cr_arrow.cu): for side s, the
// eigen-decomposition of [diag(d) z; z^T alpha] (d: n ascending, alpha a device
// scalar) into mu (n + 1, ascending; may alias d) and W ((n + 1)^2, ld n + 1).
// work: 2 * arrow_work_doubles(nmax) doubles.
size_t arrow_work_doubles(int nmax);
cudaError_t arrow_update(int n, int nmax, const double* const d[2], const double* const z[2],
                         const double* const alpha[2], double* const mu[2], double* const W[2], double* work,
                         cudaStream_t st);
// Diagonal of the eigenbasis Galerkin operator with each G_a replaced by its mean
// diagonal g_a = tr(G_a) / j (g: m doubles, written):
//   Dl(i, k) = lam (A2t_ii + 2 la_i lb_k + B2t_kk),  Den = Dl + sum_a g_a Ht(k, a)^2,
//   Hg = Ht diag(sqrt g)  (ld x m)
void galerkin_eig_diag(int j, int m, int64_t ld, double lam, const double* A2t, const double* B2t, const double* la,
                       const double* lb, const double* G, const double* Ht, double* g, double* Den, double* Dl,
                       double* Hg, cudaStream_t st);
// Ci: j blocks of m x m, C_i^-1 with C_i = I + Hg^T diag(1 / Dl(i, :)) Hg.
// cudaErrorNotSupported for m > 128.
cudaError_t galerkin_smw_setup(int j, int m, int64_t ld, const double* Dl, const double* Hg, double* Ci,
                               cudaStream_t st);
// T = double (float64 form) or float (inner solve of the mixed form); eig = nullptr: original basis
template <class T>
cudaError_t galerkin_cg_launch(int nb, int j, int m, int64_t ld, double lam, const T* A1, const T* A2, const T* B1,
                               const T* B2, const T* G, const T* H, const T* F, const T* Dg, T* Z, T* R, T* Pa,
                               T* Pb, T* Q, T* T2, T* T1, T* TH, T* Gw, T* zb, double* part, unsigned* bar,
                               int* err, double tol2, int maxit, double* out, cudaStream_t st,
                               const GalEig<T>* eig = nullptr);

// Single-cluster float32 Galerkin CG (inner solves of the mixed form, j <= 128,
// m <= 128); cudaErrorNotSupported when the sizes do not fit.  Solves
// K32 Z = F from Z = 0 until |F - K32 Z|^2 <= tol2.  out: iterations, |R|^2, status.
// eig != nullptr: the eigenbasis form (Qa, la, lb used; A2, B2, H, Dg transformed).
cudaError_t galerkin_cluster_f32_launch(int j, int m, int64_t ld, double lam, const float* A1, const float* A2,
                                        const float* B1, const float* B2, const float* G, const float* H,
                                        const float* F, const float* Dg, float* Z, double tol2, int maxit,
                                        double* out, cudaStream_t st, const GalEig<float>* eig = nullptr);

// ---------------------------------------------------------------- cr_net.cu / cr_fcg.cu
cudaError_t net_apply(cr_net* n, const float* in, float* out, cudaStream_t st);
int64_t net_voxels(const cr_net* n);
void fcg_jacobi_diag(const DevLap& L, double lam, const double* coef, int side, int m, const uint8_t* Om, int64_t ldo,
                     const double* xi, const DevXLocal& X, const double* s, double* omt, double* dinv,
                     cudaStream_t st);
void fcg_apply(const DevLap& L, double lam, const double* coef, int side, const double* omt, const DevXLocal& X,
               const int* xc_ptr, const int* xc_row, const double* xc_val, int m, const double* s, double* y,
               const double* p, double* t, double* out, cudaStream_t st);
void fcg_precond(int n, const int* box, const double* dinv, const double* r, double* s2, float* in, int64_t V,
                 cr_net* net, float* out, double* z, cudaStream_t st);
void fcg_update_xr(int n, double* x, double* r, double* rold, const double* p, const double* q, const double* sc,
                   cudaStream_t st);
void fcg_diff(int n, const double* r, const double* rold, double* d, cudaStream_t st);
void fcg_update_p(int n, double* p, const double* z, const double* sc, cudaStream_t st);

// ---------------------------------------------------------------- cr_tc.cu
size_t tc_part_elems(int splits, int m);
void bf16_split(int n, int cols, const double* U, int64_t ldu, void* hi, void* lo, int64_t ldb, cudaStream_t st);
cudaError_t galerkin_assemble_tc(int n, int j, int m, const void* hi, const void* lo, int64_t ldb, const uint8_t* Om,
                                 int64_t ldo, int splits, float* part, float* G, int64_t ld, int* err,
                                 cudaStream_t st);

}  // namespace cr

namespace cr {
// ---------------------------------------------------------------- cr_small.cu
// g[3p+s] = coef_s * sum_q Zop(p, q) h[3q + 2 - s], coef = (lam, 2 lam, lam), Zop = Z or Z^T
void zcoef(int j, const double* Z, int64_t ldz, int trans, const double* h, double lam, double* g, cudaStream_t st);
// A(col, p) = A(p, col) for p < col, in `batch` matrices spaced `stride` apart
void mirror_col(int col, double* A, int64_t ld, int batch, int64_t stride, cudaStream_t st);
// Z(j, q) = Z(q, j) = 0 for q <= j
void zero_border(int j, double* Z, int64_t ld, cudaStream_t st);
// E = OmY - Om o E  (ny x m, ld ny)
void mask_residual(int n, int m, const double* OmY, const uint8_t* Om, int64_t ldo, double* E, cudaStream_t st);
// B(i, a) = Om(i, a) * u(i)
void omega_times(int n, int m, const uint8_t* Om, int64_t ldo, const double* u, double* B, cudaStream_t st);
// out[0] = sum_{i<r, l<c} A(i,l) B(i,l) (single deterministic reduction)
void mat_dot(int r, int c, const double* A, int64_t lda, const double* B, int64_t ldb, double* out, cudaStream_t st);
// out[0] = sum Om (P - Y)^2, out[1] = sum Om Y^2 over n x m (P, Y, Om contiguous, ld n)
void cv_err(int n, int m, const double* P, const double* Y, const uint8_t* Om, double* out, cudaStream_t st);

// ---------------------------------------------------------------- cr_post.cu
// Statistics of the solution pass, in slot order: count of negative entries of
// W, min and max entry, |W|^2, |min(0, W)|^2, |W*|^2, |P(W) - W*|^2, max |P(W) - W*|.
enum { PS_NNEG, PS_MIN, PS_MAX, PS_W2, PS_NEG2, PS_REF2, PS_DIFF2, PS_MAXABS, PS_N };
// resident CTAs of the pass on this GPU; partial rows of one post_tiles launch
int post_blocks();
int post_tiles_parts(int ny, int ncols);
// Columns [col0, col0 + ncols) of W = P V^T (P = U Z: ny x j, ld ldp; V(c, k) at
// V[c + k ldv]) against W* = Pr Vr^T (jr = 0: W* = 0); P(W) = max(0, W) if nonneg.
// Writes post_tiles_parts(ny, ncols) rows of PS_N statistics to part, and P(W)
// to out (column c at out + (c - col0) ldo) unless out is null.
void post_tiles(int ny, int j, const double* P, int64_t ldp, const double* V, int64_t ldv, int jr,
                const double* Pr, int64_t ldpr, const double* Vr, int64_t ldvr, int nonneg, int col0, int ncols,
                double* out, int64_t ldo, double* part, cudaStream_t st);
// out[0..PS_N) = the fixed-order combination of nparts rows of statistics
void post_reduce(int nparts, const double* part, double* out, cudaStream_t st);
// out[0] = |Z - Zp|_F^2, out[1] = |Z|_F^2 over j x j
void mat_diff_norms(int j, const double* Z, const double* Zp, int64_t ld, double* out, cudaStream_t st);
// C = alpha A + beta B (r x c); B may alias C
void mat_axpby(int r, int c, double alpha, const double* A, int64_t lda, double beta, const double* B, int64_t ldb,
               double* C, int64_t ldc, cudaStream_t st);
// dst(i, l) = src(i, l)
void copy2d(int r, int c, const double* src, int64_t lds, double* dst, int64_t ldd, cudaStream_t st);
// Galerkin CG updates with device scalars gs: rho_k = gs[k & 1], pq = gs[2]
void cg_update_zr(int j, double* Z, double* R, const double* P, const double* Q, int64_t ld, const double* gs, int k,
                  cudaStream_t st);
void cg_update_p(int j, double* P, const double* R, int64_t ld, const double* gs, int k, cudaStream_t st);
// Dg(p, q) = diagonal of the projected operator at Z(p, q) (Jacobi preconditioner of the Galerkin CG)
void galerkin_diag(int j, int m, const double* A1, const double* A2, const double* B1, const double* B2,
                   const double* G, const double* H, int64_t ld, double lam, double* Dg, cudaStream_t st);
// y[i] = (float) x[i]
void to_f32(int64_t n, const double* x, float* y, cudaStream_t st);
// y(i, l) += (double) x(i, l)
void add_f32(int r, int c, const float* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st);
// Zp = R ./ Dg, out0 = <R, Zp>, out1 = <R, R>
void precond_dots(int j, const double* R, const double* Dg, int64_t ld, double* Zp, double* out0, double* out1,
                  cudaStream_t st);
}  // namespace cr
