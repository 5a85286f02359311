// C ABI of libconreg: problem set-up and the host-side driver of Algorithm 1
// (greedy rank-1 ALS updates, orthogonalisation, Galerkin projection,
// residual).  Every numerical step runs in the kernels of cr_pcg.cu,
// cr_blas.cu and cr_small.cu on the problem's stream; the host only sequences
// launches and reads back the few scalars that decide control flow (the ALS
// test, the Galerkin CG test, the stopping test).
//
// Residual products without forming R_j (Sec. 2.3, right sides of Eqs.
// ALS_linsys / ALS_linsys_v).  For W = U Z V^T,
//   R_j v   = E (X^T v) - lam [U Z (V^T L_x^2 v) + 2 L_yU Z (V^T L_x v) + L_y^2 U Z (V^T v)]
//   R_j^T u = X (E^T u) - lam [L_x^2 V Z^T (U^T u) + 2 L_xV Z^T (U^T L_y u) + V Z^T (U^T L_y^2 u)]
// with E = Omega o (Y - U Z V^T X), because D - C(W) = (Omega o (Y - W X)) X^T.
// With the interleaved panels UU = [u_p, L u_p, L^2 u_p]_p and VV likewise each
// product is E-times-vector plus one panel-times-vector with a 3j coefficient
// vector (zcoef).
//
// Residual norm (Algorithm 1's residual; relative Frobenius norm).  R is never
// formed: R = [E | UU] M [X | VV]^T with a block core M (the identity on the m
// data columns; for the panel block (3p+s, 3q+t): -lam Z(p,q) for (s,t) = (0,2)
// and (2,0), -2 lam Z(p,q) for (1,1); do_relres applies it without forming it).  With
// orthonormal bases Q_P of span[E | UU] and Q_Q of span[X | VV] and C_P = Q_P^T
// [E | UU], C_Q = Q_Q^T [X | VV], ||R||_F = ||C_P M C_Q^T||_F.  The bases of
// UU, X and VV grow by Gram-Schmidt as columns are appended; only E (m columns)
// is re-orthogonalised at each evaluation.  Nothing is squared, so the norm is
// accurate far below the 1e-6 relative level (a Gram-matrix formula would lose
// half the digits to cancellation).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "conreg.h"
#include "cr_common.cuh"
#include "cr_host_linalg.h"
#include "cr_mg_host.h"

using cr_host::jacobi_svd;
using cr_host::sym_eig;

using namespace cr;

namespace {
thread_local std::string g_create_err;

// Mixed form: relative residual each float32 inner PCG solve of a refinement
// step aims for (float32 vectors resolve little below 1e-6), and the cap on
// refinement steps before the float64 kernel takes over.
constexpr double kMixedInnerTol = 1e-5;
constexpr int kMaxRefine = 8;

enum {
  DS_UN2 = 0, DS_VN2 = 1, DS_NB = 2, DS_NA = 3, DS_DW = 4, /*5*/ DS_ZKZ = 6, DS_ZF = 7, DS_RN = 8, DS_V0 = 9,
  DS_GS = 16, DS_FCG = 24, DS_REF = 30, DS_COUNT = 32
};

struct HostScal {
  PcgStat stat[2];
  double ds[DS_COUNT];
};
}  // namespace

namespace cr {
// Error text reported by cr_last_error(NULL) for calls without a problem handle.
void set_global_error(const std::string& msg) { g_create_err = msg; }

// A descriptor whose arrays are device memory (mem_kind = CR_MEM_DEVICE),
// staged into host vectors: *view points into *store with mem_kind = host.  A
// host descriptor is passed through unchanged.
cr_status stage_desc(const cr_problem_desc* d, DescCopy* store, cr_problem_desc* view, std::string& err) {
  *view = *d;
  if (d->mem_kind == CR_MEM_HOST) return CR_OK;
  if (d->mem_kind != CR_MEM_DEVICE) {
    err = "mem_kind must be CR_MEM_HOST or CR_MEM_DEVICE";
    return CR_EINVAL;
  }
  const int64_t nx = d->nx, ny = d->ny, m = d->ninj;
  if (nx <= 0 || ny <= 0 || m <= 0 || nx > (1 << 24) || ny > (1 << 24) || m > 4096 || d->ldx < nx || d->ldy < ny ||
      d->ldo < ny || d->Lx.n != nx || d->Ly.n != ny) {
    err = "bad sizes";
    return CR_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    err = "no current CUDA device";
    return CR_ECUDA;
  }
  auto on_device = [&](const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
  };
  const void* ptrs[] = {d->Lx.rowptr, d->Lx.col, d->Lx.val, d->Ly.rowptr, d->Ly.col, d->Ly.val,
                        d->X_host,    d->Y_host, d->Omega_host};
  for (const void* q : ptrs)
    if (!on_device(q)) {
      err = "mem_kind = CR_MEM_DEVICE but an array is not device memory of the current GPU";
      return CR_EINVAL;
    }
  auto get = [&](void* dst, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
  };
  bool ok = true;
  for (int side = 0; side < 2 && ok; ++side) {
    const cr_csr& c = side == 0 ? d->Lx : d->Ly;
    std::vector<int32_t>& rp = side == 0 ? store->lx_rp : store->ly_rp;
    std::vector<int32_t>& col = side == 0 ? store->lx_col : store->ly_col;
    std::vector<double>& val = side == 0 ? store->lx_val : store->ly_val;
    rp.resize((size_t)c.n + 1);
    ok = get(rp.data(), c.rowptr, sizeof(int32_t) * rp.size());
    if (ok && (rp[0] != 0 || rp[c.n] < 0 || rp[c.n] > (int32_t)((c.n) * 17))) {
      err = "bad CSR row pointers";
      return CR_EINVAL;
    }
    if (ok) {
      col.resize((size_t)rp[c.n]);
      val.resize((size_t)rp[c.n]);
      ok = get(col.data(), c.col, sizeof(int32_t) * col.size()) && get(val.data(), c.val, sizeof(double) * val.size());
    }
    cr_csr& vc = side == 0 ? view->Lx : view->Ly;
    vc.rowptr = rp.data();
    vc.col = col.data();
    vc.val = val.data();
  }
  store->X.resize((size_t)nx * m);
  store->Y.resize((size_t)ny * m);
  store->Om.resize((size_t)ny * m);
  ok = ok && cudaMemcpy2D(store->X.data(), nx * sizeof(double), d->X_host, d->ldx * sizeof(double), nx * sizeof(double),
                          m, cudaMemcpyDeviceToHost) == cudaSuccess;
  ok = ok && cudaMemcpy2D(store->Y.data(), ny * sizeof(double), d->Y_host, d->ldy * sizeof(double), ny * sizeof(double),
                          m, cudaMemcpyDeviceToHost) == cudaSuccess;
  ok = ok && cudaMemcpy2D(store->Om.data(), ny, d->Omega_host, d->ldo, ny, m, cudaMemcpyDeviceToHost) == cudaSuccess;
  for (int side = 0; side < 2 && ok; ++side) {
    const cr_grid& g = side == 0 ? d->grid_x : d->grid_y;
    if (!g.box_index) continue;
    if (!on_device(g.box_index)) {
      err = "mem_kind = CR_MEM_DEVICE but a grid's box indices are not device memory of the current GPU";
      return CR_EINVAL;
    }
    std::vector<int32_t>& b = side == 0 ? store->gx : store->gy;
    b.resize((size_t)(side == 0 ? nx : ny));
    ok = get(b.data(), g.box_index, sizeof(int32_t) * b.size());
    (side == 0 ? view->grid_x : view->grid_y).box_index = b.data();
  }
  if (!ok) {
    err = std::string("staging device inputs failed: ") + cudaGetErrorString(cudaGetLastError());
    return CR_ECUDA;
  }
  view->X_host = store->X.data();
  view->ldx = nx;
  view->Y_host = store->Y.data();
  view->ldy = ny;
  view->Omega_host = store->Om.data();
  view->ldo = ny;
  view->mem_kind = CR_MEM_HOST;
  return CR_OK;
}
}  // namespace cr

struct cr_problem;
namespace cr {
cr_status adopt_stream(cr_problem* p, cudaStream_t st);
}

struct cr_problem {
  int nx = 0, ny = 0, m = 0, rcap = 0;
  double lam = 0.0;
  cr_options opt{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  int j = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  DevLap Lx, Ly;
  DevMg mg[2];  // multigrid hierarchies of L_y (side 0) and L_x (side 1)
  int *xc_ptr = nullptr, *xc_row = nullptr;
  double* xc_val = nullptr;
  DevXLocal xl;
  double* OmY = nullptr;
  uint8_t* Om = nullptr;
  double *UU = nullptr, *VV = nullptr, *Z = nullptr, *Zprev = nullptr;
  double *A1 = nullptr, *A2 = nullptr, *B1 = nullptr, *B2 = nullptr, *H = nullptr, *P = nullptr, *G = nullptr,
         *F = nullptr, *E = nullptr, *Mzh = nullptr;
  double *u = nullptr, *v = nullptr, *uhat = nullptr, *vhat = nullptr, *rhs_u = nullptr, *rhs_v = nullptr;
  double *tmpy = nullptr, *tmpx = nullptr, *xi = nullptr, *eta = nullptr, *svec = nullptr, *hc = nullptr,
         *gc = nullptr, *coef = nullptr, *cvec = nullptr, *Bnm = nullptr;
  double *pr = nullptr, *pp = nullptr, *ps = nullptr, *pw = nullptr, *pdinv = nullptr, *pomt = nullptr;
  PcgStat* stat = nullptr;
  double* ds = nullptr;
  HostScal* hs = nullptr;  // pinned
  double *gR = nullptr, *gP = nullptr, *gQ = nullptr, *gZB2 = nullptr, *gZB1 = nullptr, *gZH = nullptr,
         *gGw = nullptr, *gDg = nullptr, *gT = nullptr, *gzb = nullptr, *gpart = nullptr, *gout = nullptr;
  unsigned* gbar = nullptr;
  int* gerr = nullptr;
  int gal_nb = 0;
  // Galerkin CG in the eigenbasis of A1 and B1: eigenvectors Qa, Qb (each with a
  // second buffer for the update; zero outside the leading eq x eq block),
  // eigenvalues (host and device), transformed matrices and work.  eq = borders
  // taken into the bases so far.
  double *eQa = nullptr, *eQa2 = nullptr, *eQb = nullptr, *eQb2 = nullptr, *ela = nullptr, *elb = nullptr;
  double *eA2t = nullptr, *eB2t = nullptr, *eFt = nullptr, *eZt = nullptr, *eDen = nullptr, *eTmp = nullptr;
  double *eHt = nullptr, *eY = nullptr, *eGt = nullptr, *eg = nullptr, *eW = nullptr, *ebord = nullptr;
  double* earw = nullptr;  // arrowhead work, both sides
  // row-wise Sherman-Morrison-Woodbury preconditioner of the eigenbasis CG (m <= 128)
  double *eDl = nullptr, *eHg = nullptr, *eCi = nullptr, *eS = nullptr, *eZz = nullptr, *eYd = nullptr;
  bool smw_ok = false;  // set per projection when the capacitance inverses are ready
  float *fQa = nullptr, *fla = nullptr, *flb = nullptr, *fY = nullptr, *fGt = nullptr;
  float* fZz = nullptr;
  int eq = 0;
  int64_t gal_eig_proj = 0, gal_eig_finish = 0;
  // float32 copies for the mixed form's inner Galerkin CG
  // learned preconditioner: box index of each row per side, the network, its buffers
  int* box[2] = {nullptr, nullptr};
  int box_dims[2][3] = {{0, 0, 0}, {0, 0, 0}};
  cr_net* net = nullptr;
  float *net_in = nullptr, *net_out = nullptr;
  int64_t net_V = 0;
  double *fc_rold = nullptr, *fc_d = nullptr, *fc_t = nullptr, *fc_y = nullptr;
  // held-out scoring (cr_cv_error): buffers for cv_cap columns
  int cv_cap = 0;
  double *cv_X = nullptr, *cv_Y = nullptr, *cv_T1 = nullptr, *cv_T2 = nullptr, *cv_P = nullptr, *cv_out = nullptr;
  uint8_t* cv_Om = nullptr;
  // post-processing (cr_svd_factors, cr_solution_report): P = U Z, reference factors
  // for post_ref_cap columns, the statistics' partial rows, a column block of W
  double *post_P = nullptr, *post_part = nullptr, *post_out = nullptr, *post_W = nullptr;
  double *post_Ur = nullptr, *post_Zr = nullptr, *post_Vr = nullptr, *post_Pr = nullptr;
  double *post_small = nullptr, *post_Uh = nullptr, *post_Vh = nullptr;
  int post_ref_cap = 0;
  int64_t post_part_cap = 0, post_W_cols = 0;
  int64_t fcg_fallbacks = 0, learned_solves = 0, mixed_handovers = 0;
  // grid-wide PCG (grids the register-resident kernel does not take, or pcg_kernel = 2): work buffers
  double *pg_work = nullptr, *pg_part = nullptr, *pg_ypart = nullptr, *pg_yglob = nullptr;
  unsigned* pg_bar = nullptr;
  int* pg_err = nullptr;
  // Jacobi as judge of the learned preconditioner, per side: the iteration count of
  // a Jacobi-PCG solve (0 = not measured yet), consecutive fallbacks, and whether
  // the learned form has been switched off for this side
  int jac_iters[2] = {0, 0};
  double jac_sec[2] = {0.0, 0.0};  // host time of the judge's Jacobi-PCG solve
  int learned_streak[2] = {0, 0};
  bool learned_off[2] = {false, false};
  // BF16 hi/lo shadows of U (n_y x 128, column stride ldb) for the tensor-core assembly
  void *ubhi = nullptr, *ublo = nullptr;
  int64_t ldb = 0;
  int tc_splits = 0;
  float* tcpart = nullptr;
  int* tcerr = nullptr;
  float *fA1 = nullptr, *fA2 = nullptr, *fB1 = nullptr, *fB2 = nullptr, *fDg = nullptr, *fH = nullptr,
        *fG = nullptr, *fF = nullptr, *fZ = nullptr, *fR = nullptr, *fPa = nullptr, *fPb = nullptr, *fQ = nullptr,
        *fT2 = nullptr, *fT1 = nullptr, *fTH = nullptr, *fGw = nullptr, *fzb = nullptr;
  double *QL = nullptr, *CL = nullptr, *QR = nullptr, *CRm = nullptr, *Cx = nullptr, *Cx2 = nullptr, *Ep = nullptr,
         *CE = nullptr, *CP = nullptr, *T1 = nullptr, *T2 = nullptr, *gram = nullptr, *tmat = nullptr;
  int nQL = 0, nQR = 0, nQX = 0;
  std::vector<int> qr_step;  // greedy step that created right-basis vector nQX + i
  int64_t ldcl = 0, ldcr = 0, ldcx = 0, ldcp = 0, ldm = 0;
  double* ws = nullptr;
  size_t ws_elems = 0;
  double Dnorm = 0.0, OmYn2 = 0.0;
  bool F_valid = false;
  double last_dW = NAN;
  // profiling
  struct Pending {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Pending> pending;
  cudaEvent_t open_ev[CR_NPHASE] = {};
  double phase_ms[CR_NPHASE] = {};
  int64_t phase_calls[CR_NPHASE] = {};
  int64_t pcg_solves = 0, pcg_iters = 0, pcg_iters_side[2] = {0, 0};
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  long long launch_base = 0;
};

namespace {

#define CUCHK(p, x)                                                                                   \
  do {                                                                                                \
    cudaError_t e_ = (x);                                                                             \
    if (e_ != cudaSuccess) {                                                                          \
      (p)->err = std::string(#x) + " failed: " + cudaGetErrorString(e_);                              \
      return CR_ECUDA;                                                                                \
    }                                                                                                 \
  } while (0)

#define TRY(x)                         \
  do {                                 \
    cr_status s_ = (x);                \
    if (s_ != CR_OK) return s_;        \
  } while (0)

cudaEvent_t take_event(cr_problem* p) {
  if (!p->ev_pool.empty()) {
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(cr_problem* p, int ph) {
  if (!p->opt.profile) return;
  cudaEvent_t e = take_event(p);
  cudaEventRecord(e, p->st);
  p->open_ev[ph] = e;
}

void prof_end(cr_problem* p, int ph) {
  if (!p->opt.profile || !p->open_ev[ph]) return;
  cudaEvent_t e = take_event(p);
  cudaEventRecord(e, p->st);
  p->pending.push_back({ph, p->open_ev[ph], e});
  p->open_ev[ph] = nullptr;
}

void prof_resolve(cr_problem* p) {
  for (auto& q : p->pending) {
    float ms = 0.0f;
    cudaEventSynchronize(q.b);
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      p->phase_ms[q.phase] += ms;
      p->phase_calls[q.phase] += 1;
    }
    p->ev_pool.push_back(q.a);
    p->ev_pool.push_back(q.b);
  }
  p->pending.clear();
  cudaGetLastError();
}

cr_status fail(cr_problem* p, cr_status s, const std::string& msg) {
  p->err = msg;
  return s;
}

template <class T>
cr_status dalloc(cr_problem* p, T** out, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  void* ptr = nullptr;
  if (p->opt.alloc) {
    ptr = p->opt.alloc(bytes, p->opt.alloc_ctx);
    if (!ptr) return fail(p, CR_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  } else {
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(p, CR_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
  }
  p->allocs.push_back({ptr, bytes});
  *out = static_cast<T*>(ptr);
  CUCHK(p, cudaMemsetAsync(ptr, 0, bytes, p->st));
  return CR_OK;
}

template <class T>
cr_status upload(cr_problem* p, T** out, const std::vector<T>& h) {
  TRY(dalloc(p, out, h.size()));
  if (!h.empty()) CUCHK(p, cudaMemcpyAsync(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, p->st));
  p->h2d_bytes += (int64_t)(h.size() * sizeof(T));
  return CR_OK;
}

cr_status sync(cr_problem* p) {
  CUCHK(p, cudaGetLastError());
  CUCHK(p, cudaStreamSynchronize(p->st));
  return CR_OK;
}

// Read device scalars ds[lo..lo+cnt) and both PCG stats into the pinned mirror.
cr_status readback(cr_problem* p, int lo, int cnt, bool stats) {
  CUCHK(p, cudaMemcpyAsync(p->hs->ds + lo, p->ds + lo, sizeof(double) * cnt, cudaMemcpyDeviceToHost, p->st));
  p->d2h_bytes += (int64_t)(sizeof(double) * cnt);
  if (stats) {
    CUCHK(p, cudaMemcpyAsync(p->hs->stat, p->stat, sizeof(PcgStat) * 2, cudaMemcpyDeviceToHost, p->st));
    p->d2h_bytes += (int64_t)(sizeof(PcgStat) * 2);
  }
  return sync(p);
}

// --------------------------------------------------------------------------- set-up helpers
// Box indices of one side: distinct and inside the D x H x W box.
bool grid_ok(const int32_t* dims, const int32_t* idx, int64_t n, std::string& err) {
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (int64_t)dims[0] * dims[1] * dims[2] > (1ll << 26)) {
    err = "bad box dimensions";
    return false;
  }
  const int64_t V = (int64_t)dims[0] * dims[1] * dims[2];
  std::vector<uint8_t> seen((size_t)V, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (idx[i] < 0 || idx[i] >= V || seen[idx[i]]) {
      err = "box indices out of range or repeated";
      return false;
    }
    seen[idx[i]] = 1;
  }
  return true;
}

struct HostCSR {
  int64_t n;
  std::vector<int32_t> rp, col;
  std::vector<double> val;
};

cr_status check_csr(const cr_csr& c, int64_t n, const char* name, std::string& err) {
  if (c.n != n || !c.rowptr || !c.col || !c.val) {
    err = std::string(name) + ": size mismatch or null pointer";
    return CR_EINVAL;
  }
  if (c.rowptr[0] != 0) {
    err = std::string(name) + ": rowptr[0] != 0";
    return CR_EINVAL;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (c.rowptr[i + 1] < c.rowptr[i]) {
      err = std::string(name) + ": rowptr not monotone";
      return CR_EINVAL;
    }
    int off = 0;
    for (int32_t q = c.rowptr[i]; q < c.rowptr[i + 1]; ++q) {
      if (c.col[q] < 0 || c.col[q] >= n || !std::isfinite(c.val[q])) {
        err = std::string(name) + ": bad column index or non-finite value in row " + std::to_string(i);
        return CR_EINVAL;
      }
      if (c.col[q] != i && c.val[q] != 0.0) ++off;
    }
    if (off > kMaxSlots) {
      err = std::string(name) + ": more than 16 off-diagonal entries in row " + std::to_string(i);
      return CR_EINVAL;
    }
  }
  // symmetry: compare the entry list with its transpose
  std::vector<std::tuple<int32_t, int32_t, double>> a, b;
  const int64_t nnz = c.rowptr[n];
  a.reserve(nnz);
  b.reserve(nnz);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t q = c.rowptr[i]; q < c.rowptr[i + 1]; ++q)
      if (c.val[q] != 0.0) {
        a.emplace_back((int32_t)i, c.col[q], c.val[q]);
        b.emplace_back(c.col[q], (int32_t)i, c.val[q]);
      }
  std::sort(a.begin(), a.end());
  std::sort(b.begin(), b.end());
  if (a != b) {
    err = std::string(name) + ": matrix is not symmetric";
    return CR_EINVAL;
  }
  return CR_OK;
}

// Build the padded ELL layout and the PCG partition of one Laplacian.
cr_status build_lap(cr_problem* p, const cr_csr& c, DevLap& L) {
  const int n = (int)c.n;
  std::vector<double> diag(n, 0.0), l2(n, 0.0);
  std::vector<std::vector<std::pair<int, double>>> rows(n);
  bool unit = true;
  int K = 1;
  for (int i = 0; i < n; ++i) {
    for (int32_t q = c.rowptr[i]; q < c.rowptr[i + 1]; ++q) {
      const int jj = c.col[q];
      const double v = c.val[q];
      if (jj == i) {
        diag[i] += v;
      } else if (v != 0.0) {
        rows[i].push_back({jj, v});
        if (v != -1.0) unit = false;
      }
    }
    // merge duplicate columns
    std::sort(rows[i].begin(), rows[i].end());
    std::vector<std::pair<int, double>> merged;
    for (auto& e : rows[i]) {
      if (!merged.empty() && merged.back().first == e.first)
        merged.back().second += e.second;
      else
        merged.push_back(e);
    }
    rows[i] = merged;
    for (auto& e : rows[i])
      if (e.second != -1.0) unit = false;
    K = std::max<int>(K, (int)rows[i].size());
  }
  for (int i = 0; i < n; ++i) {
    double s = diag[i] * diag[i];
    for (auto& e : rows[i]) s += e.second * e.second;
    l2[i] = s;
  }
  // partition for the cluster PCG
  const size_t smem_cap = 227 * 1024;
  int desired = std::min(kMaxCluster, std::max(1, (n + 479) / 480));
  int cs = 0, chunk = 0;
  for (int c2 = desired; c2 >= 1; --c2) {
    const int ch = (n + c2 - 1) / c2;
    const size_t smem = pcg_smem_bytes(ch, p->m);
    if (smem > smem_cap) break;
    if (pcg_cluster_ok(c2, smem)) {
      cs = c2;
      chunk = ch;
      break;
    }
  }
  if (cs == 0) {
    // too large for one cluster: the sub-solves run on the grid-wide PCG
    chunk = n;
  } else if (p->opt.cluster_size > 0 && p->opt.cluster_size != cs && p->opt.cluster_size <= kMaxCluster &&
             p->opt.cluster_size <= n) {
    // a requested cluster size replaces the automatic one when the chunks fit
    // (smaller or larger than automatic; CTAs past the last row hold no rows)
    const int c2 = p->opt.cluster_size;
    const int ch = (n + c2 - 1) / c2;
    if (pcg_smem_bytes(ch, p->m) <= smem_cap && pcg_cluster_ok(c2, pcg_smem_bytes(ch, p->m))) {
      cs = c2;
      chunk = ch;
    }
  }
  std::vector<int> nbr((size_t)K * n, -1), nbrp((size_t)K * n, -1);
  std::vector<double> offw(unit ? 0 : (size_t)K * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (size_t k = 0; k < rows[i].size(); ++k) {
      const int jj = rows[i][k].first;
      nbr[k * n + i] = jj;
      nbrp[k * n + i] = ((jj / chunk) << 24) | (jj % chunk);
      if (!unit) offw[k * n + i] = rows[i][k].second;
    }
  int *dn = nullptr, *dnp = nullptr;
  double *dd = nullptr, *dl2 = nullptr, *dw = nullptr;
  TRY(upload(p, &dn, nbr));
  TRY(upload(p, &dnp, nbrp));
  TRY(upload(p, &dd, diag));
  TRY(upload(p, &dl2, l2));
  if (!unit) TRY(upload(p, &dw, offw));
  L.n = n;
  L.K = K;
  L.nbr = dn;
  L.nbrp = dnp;
  L.offw = dw;
  L.diag = dd;
  L.l2diag = dl2;
  L.chunk = chunk;
  L.csize = cs;
  if (cs > 0) CUCHK(p, pcg_prepare(0, cs, pcg_smem_bytes(chunk, p->m)));
  return CR_OK;
}

// Multigrid hierarchy of one Laplacian (cr_mg_host.h) on the cluster partition
// of L: level 0 in L's chunks, larger coarse levels in equal chunks over the
// cluster, levels of at most kMgTailRows rows and the coarsest (at most
// kMgCoarseMax rows, through the eigenbasis of its pencil) on CTA 0.  Leaves
// g.nlev = 0 when the hierarchy or its shared memory does not fit.
cr_status build_mg(cr_problem* p, const cr_csr& c, const DevLap& L, DevMg& g) {
  g = DevMg{};
  const int n = (int)c.n;
  const int C = L.csize;
  if (C < 1 || n <= kMgCoarseMax) return CR_OK;
  cr_mg::Csr A;
  A.rows = A.cols = n;
  A.rp.assign(n + 1, 0);
  std::vector<std::pair<int, double>> row;
  for (int i = 0; i < n; ++i) {
    row.clear();
    for (int32_t q = c.rowptr[i]; q < c.rowptr[i + 1]; ++q) row.push_back({c.col[q], c.val[q]});
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) {
      if (!A.ci.empty() && (int)A.ci.size() > A.rp[i] && A.ci.back() == row[k].first)
        A.v.back() += row[k].second;
      else {
        A.ci.push_back(row[k].first);
        A.v.push_back(row[k].second);
      }
    }
    A.rp[i + 1] = (int)A.ci.size();
  }
  const cr_mg::Hierarchy H = cr_mg::build(A, kMgCoarseMax, kMgMaxLev);
  const int nlev = (int)H.lev.size();
  if (nlev < 2 || H.lev.back().L.rows > kMgCoarseMax) return CR_OK;
  double bytes_iter[2];
  for (int wi = 0; wi < 2; ++wi) {
    const double w = wi == 0 ? 4.0 : 8.0;
    double vc = 0.0;
    for (int l = 0; l + 1 < nlev; ++l) {
      const cr_mg::Level& HL = H.lev[l];
      const double nl = HL.L.rows;
      vc += 4.0 * ((double)HL.L.nnz() * (4.0 + w) + 3.0 * nl * w) +
            (double)(HL.P.nnz() + HL.R.nnz()) * (4.0 + w) + 2.0 * nl * w;
    }
    const double ncd = H.lev.back().L.rows;
    vc += 2.0 * ncd * ncd * 8.0;
    bytes_iter[wi] = (double)n * (10.0 * w + 4.0 * L.K) + 2.0 * vc;
  }
  std::vector<double> Q, mu;
  if (!cr_mg::pencil_basis(H.lev.back().L, H.lev.back().M, Q, mu)) return CR_OK;
  DevMg h{};
  h.bytes_iter[0] = bytes_iter[0];
  h.bytes_iter[1] = bytes_iter[1];
  h.nlev = nlev;
  h.nc = H.lev.back().L.rows;
  h.ld = nlev - 1;
  int off = 0;
  for (int l = 0; l < nlev; ++l) {
    DevMgLevel& V = h.lev[l];
    V.n = H.lev[l].L.rows;
    if (l == 0) {
      V.dist = 1;
      V.chunk = L.chunk;
    } else {
      V.dist = (l < nlev - 1 && V.n > kMgTailRows && C > 1) ? 1 : 0;
      V.chunk = V.dist ? (V.n + C - 1) / C : V.n;
      V.off = off;
      off += 5 * V.chunk;
    }
  }
  for (int l = 1; l < nlev; ++l)
    if (!h.lev[l].dist) {
      h.ld = l;
      break;
    }
  h.lvl_elems = off;
  auto pack = [&](int l, int row) -> int {
    const DevMgLevel& V = h.lev[l];
    if (!V.dist) return row;
    return ((row / V.chunk) << 24) | (row % V.chunk);
  };
  for (int l = 0; l < nlev; ++l) {
    DevMgLevel& V = h.lev[l];
    const cr_mg::Level& HL = H.lev[l];
    if (l >= 1) {
      // L_l + sigma M_l on the union of both patterns (the coarsest level's too, though
      // its solve goes through the eigenbasis: every level's arrays exist)
      std::vector<int> rp(V.n + 1, 0), cp;
      std::vector<double> lv, mv, dl(V.n, 0.0), dm(V.n, 0.0);
      for (int i = 0; i < V.n; ++i) {
        int a = HL.L.rp[i], b = HL.M.rp[i];
        const int ae = HL.L.rp[i + 1], be = HL.M.rp[i + 1];
        while (a < ae || b < be) {
          const int ca = a < ae ? HL.L.ci[a] : INT32_MAX, cb = b < be ? HL.M.ci[b] : INT32_MAX;
          const int col = std::min(ca, cb);
          const double x = ca == col ? HL.L.v[a++] : 0.0;
          const double y = cb == col ? HL.M.v[b++] : 0.0;
          cp.push_back(pack(l, col));
          lv.push_back(x);
          mv.push_back(y);
          if (col == i) {
            dl[i] = x;
            dm[i] = y;
          }
        }
        rp[i + 1] = (int)cp.size();
      }
      int *drp = nullptr, *dcp = nullptr;
      double *dlv = nullptr, *dmv = nullptr, *ddl = nullptr, *ddm = nullptr;
      TRY(upload(p, &drp, rp));
      TRY(upload(p, &dcp, cp));
      TRY(upload(p, &dlv, lv));
      TRY(upload(p, &dmv, mv));
      TRY(upload(p, &ddl, dl));
      TRY(upload(p, &ddm, dm));
      V.rp = drp;
      V.cp = dcp;
      V.lv = dlv;
      V.mv = dmv;
      V.dl = ddl;
      V.dm = ddm;
    }
    if (l < nlev - 1) {
      std::vector<int> prp(HL.P.rp), pcp(HL.P.ci.size()), rrp(HL.R.rp), rcp(HL.R.ci.size());
      for (size_t q = 0; q < HL.P.ci.size(); ++q) pcp[q] = pack(l + 1, HL.P.ci[q]);
      for (size_t q = 0; q < HL.R.ci.size(); ++q) rcp[q] = pack(l, HL.R.ci[q]);
      int *d1 = nullptr, *d2 = nullptr, *d3 = nullptr, *d4 = nullptr;
      double *d5 = nullptr, *d6 = nullptr;
      TRY(upload(p, &d1, prp));
      TRY(upload(p, &d2, pcp));
      TRY(upload(p, &d5, HL.P.v));
      TRY(upload(p, &d3, rrp));
      TRY(upload(p, &d4, rcp));
      TRY(upload(p, &d6, HL.R.v));
      V.prp = d1;
      V.pcp = d2;
      V.pv = d5;
      V.rrp = d3;
      V.rcp = d4;
      V.rv = d6;
    }
  }
  double *dQ = nullptr, *dmu = nullptr;
  TRY(upload(p, &dQ, Q));
  TRY(upload(p, &dmu, mu));
  h.cQ = dQ;
  h.cmu = dmu;
  // per-CTA tables: byte layout of one CTA's sections (sizes are maxima over the CTAs)
  auto rows_of = [&](int l, int r) -> int {
    const DevMgLevel& V = h.lev[l];
    if (!V.dist) return r == 0 ? V.n : 0;
    return std::max(0, std::min(V.n - r * V.chunk, V.chunk));
  };
  auto beg_of = [&](int l, int r) -> int { return h.lev[l].dist ? r * h.lev[l].chunk : 0; };
  auto max_entries = [&](int l, const std::vector<int>& rp) -> int64_t {  // rows of level l, CSR rp
    int64_t mx = 0;
    for (int r = 0; r < C; ++r) {
      const int b = beg_of(l, r), nr = rows_of(l, r);
      if (nr > 0) mx = std::max<int64_t>(mx, rp[b + nr] - rp[b]);
    }
    return mx;
  };
  int64_t tb = 0;
  auto sect = [&](int64_t bytes) {
    const int64_t at = tb;
    tb += (bytes + 15) / 16 * 16;
    return at;
  };
  const bool unit = L.offw == nullptr;
  h.nb_a = sect(4 * (int64_t)L.K * L.chunk);
  h.nb_c = unit ? -1 : sect(8 * (int64_t)L.K * L.chunk);
  h.dg = sect(8 * (int64_t)L.chunk);
  for (int l = 0; l < nlev - 1; ++l) {
    DevMgLevel& V = h.lev[l];
    const cr_mg::Level& HL = H.lev[l];
    const int rows = l == 0 ? L.chunk : V.chunk;
    if (l >= 1) {
      // the operator rows as uploaded (union of the L and M patterns)
      std::vector<int> urp(V.n + 1, 0);
      for (int i = 0; i < V.n; ++i) {
        int a = HL.L.rp[i], b = HL.M.rp[i], cnt = 0;
        const int ae = HL.L.rp[i + 1], be = HL.M.rp[i + 1];
        while (a < ae || b < be) {
          const int ca = a < ae ? HL.L.ci[a] : INT32_MAX, cb = b < be ? HL.M.ci[b] : INT32_MAX;
          const int col = std::min(ca, cb);
          if (ca == col) ++a;
          if (cb == col) ++b;
          ++cnt;
        }
        urp[i + 1] = urp[i] + cnt;
      }
      const int64_t e = max_entries(l, urp);
      V.op_rp = sect(4 * (int64_t)(rows + 1));
      V.op_a = sect(4 * e);
      V.op_c = sect(8 * e);
    }
    const int64_t ep = max_entries(l, HL.P.rp);
    V.p_rp = sect(4 * (int64_t)(rows + 1));
    V.p_a = sect(4 * ep);
    V.p_c = sect(8 * ep);
    const int rows1 = h.lev[l + 1].chunk;
    const int64_t er = max_entries(l + 1, HL.R.rp);
    V.r_rp = sect(4 * (int64_t)(rows1 + 1));
    V.r_a = sect(4 * er);
    V.r_c = sect(8 * er);
  }
  h.tab_bytes = tb;
  h.smw = (&g == &p->mg[1] && p->m <= kMgSmwMax) ? 1 : 0;  // v side, small enough data term
  const size_t cap = 227 * 1024;
  bool need_glob = false;
  for (int f = 0; f < 2; ++f) {
    const size_t with = mg_smem_bytes(h, L.chunk, p->m, f == 0, true);
    const size_t without = mg_smem_bytes(h, L.chunk, p->m, f == 0, false);
    h.tab_smem[f] = with <= cap ? 1 : 0;
    h.smem[f] = with <= cap ? with : (without <= cap ? without : 0);
    if (h.smem[f] && !h.tab_smem[f]) need_glob = true;
  }
  if (need_glob) TRY(dalloc(p, &h.tab_glob, (size_t)C * h.tab_bytes));
  if (h.smw) {
    // the cache of the v side's Sherman-Morrison-Woodbury correction; smw_sig = {shift, precision}
    // of the MX it holds (0: none), so a launch of either precision knows whether to rebuild it
    TRY(dalloc(p, &h.smw_mx, (size_t)n * p->m));
    TRY(dalloc(p, &h.smw_xx, (size_t)p->m * p->m));
    TRY(dalloc(p, &h.smw_sig, 3));
  }
  if (h.smem[0] == 0 && h.smem[1] == 0) return CR_OK;
  CUCHK(p, mg_prepare());
  for (int f = 0; f < 2; ++f)
    if (h.smem[f] && !mg_cluster_ok(C, h.smem[f], f == 0)) h.smem[f] = 0;
  g = h;
  return CR_OK;
}

// --------------------------------------------------------------------------- device steps
// Gram-Schmidt twice: w <- w - Q (Q^T w) (x2) against Q's first nq columns,
// then w <- w / |w|.  Returns |w_after| / |w_before| (0 if w was zero).
cr_status cgs2(cr_problem* p, int n, const double* Q, int64_t ldq, int nq, double* w, double* ratio) {
  cudaStream_t st = p->st;
  dot(n, w, w, p->ds + DS_NB, st);
  for (int pass = 0; pass < 2 && nq > 0; ++pass) {
    gemv_t(n, nq, Q, ldq, w, p->cvec, 1, 1.0, 0.0, st);
    gemv_n(n, nq, Q, ldq, p->cvec, 1, w, -1.0, 1.0, st);
  }
  dot(n, w, w, p->ds + DS_NA, st);
  TRY(readback(p, DS_NB, 2, false));
  const double nb = p->hs->ds[DS_NB], na = p->hs->ds[DS_NA];
  *ratio = nb > 0.0 ? std::sqrt(na / nb) : 0.0;
  if (na > 0.0) scale_by_inv_norm(n, w, p->ds + DS_NA, w, st);
  return CR_OK;
}

// R_j v (ny entries) for v on the x grid.
void residual_times(cr_problem* p, const double* vv, double* out) {
  cudaStream_t st = p->st;
  const int j = p->j;
  spmv_xt(p->m, p->xc_ptr, p->xc_row, p->xc_val, vv, p->xi, 1, st);
  gemv_n(p->ny, p->m, p->E, p->ny, p->xi, 1, out, 1.0, 0.0, st);
  if (j > 0) {
    gemv_t(p->nx, 3 * j, p->VV, p->nx, vv, p->hc, 1, 1.0, 0.0, st);
    zcoef(j, p->Z, p->rcap, 0, p->hc, p->lam, p->gc, st);
    gemv_n(p->ny, 3 * j, p->UU, p->ny, p->gc, 1, out, -1.0, 1.0, st);
  }
}

// R_j^T u (nx entries) for u on the y grid.
void residual_t_times(cr_problem* p, const double* uu, double* out) {
  cudaStream_t st = p->st;
  const int j = p->j;
  gemv_t(p->ny, p->m, p->E, p->ny, uu, p->eta, 1, 1.0, 0.0, st);
  spmv_x(p->nx, p->xl.xr_ptr, p->xl.xr_col, p->xl.xr_val, p->eta, out, 1.0, 0.0, st);
  if (j > 0) {
    gemv_t(p->ny, 3 * j, p->UU, p->ny, uu, p->hc, 1, 1.0, 0.0, st);
    zcoef(j, p->Z, p->rcap, 1, p->hc, p->lam, p->gc, st);
    gemv_n(p->nx, 3 * j, p->VV, p->nx, p->gc, 1, out, -1.0, 1.0, st);
  }
}

// u side (Eq. ALS_linsys): coefficients c = v'L_x v, d = |L_x v|^2 and xi = X^T v.
void prep_u(cr_problem* p, const double* vv) {
  cudaStream_t st = p->st;
  lap_apply(p->Lx, vv, p->tmpx, 0.0, st);
  dot(p->nx, vv, p->tmpx, p->coef + 0, st);
  dot(p->nx, p->tmpx, p->tmpx, p->coef + 1, st);
  spmv_xt(p->m, p->xc_ptr, p->xc_row, p->xc_val, vv, p->xi, 1, st);
}

// v side (Eq. ALS_linsys_v): c' = u'L_y u, d' = |L_y u|^2, s_a = u' diag(Omega_a) u.
void prep_v(cr_problem* p, const double* uu) {
  cudaStream_t st = p->st;
  lap_apply(p->Ly, uu, p->tmpy, 0.0, st);
  dot(p->ny, uu, p->tmpy, p->coef + 2, st);
  dot(p->ny, p->tmpy, p->tmpy, p->coef + 3, st);
  omega_sq_dots(p->ny, p->m, p->Om, p->ny, uu, p->svec, st);
}

cr_status launch_pcg_jacobi(cr_problem* p, int side, const double* b, double* x, int maxit);
cr_status launch_pcg_mixed(cr_problem* p, int side, const double* b, double* x, int maxit);

// Flexible CG (Polak-Ribiere) with the learned preconditioner
// z = D^-1 r + s net(D^-1 r / s, mask); float64 vectors.  It may take at most
// 2 k_J + 16 iterations and (judging by time) 2 t_J, k_J and t_J being the
// judge's Jacobi-PCG solve on this side; if it has not converged by then,
// Jacobi-PCG continues from its iterate (fallback).  Writes the PcgStat of
// `side` like the PCG.
cr_status fcg_learned(cr_problem* p, int side, const double* b, double* x) {
  cudaStream_t st = p->st;
  const DevLap& L = side == 0 ? p->Ly : p->Lx;
  const int n = L.n;
  const double* coef = p->coef + (side == 0 ? 0 : 2);
  double* sc = p->ds + DS_FCG;
  double *r = p->pr, *q = p->pw, *pv = p->pp, *z = p->ps, *rold = p->fc_rold, *dd = p->fc_d, *t = p->fc_t;
  const double tol = p->opt.pcg_tol;
  const bool by_time = p->opt.learned_judge == 0;
  const auto t_start = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(); };
  prof_begin(p, side == 0 ? CR_PHASE_PCG_U : CR_PHASE_PCG_V);
  fcg_jacobi_diag(L, p->lam, coef, side, p->m, p->Om, p->ny, p->xi, p->xl, p->svec, p->pomt, p->pdinv, st);
  fcg_apply(L, p->lam, coef, side, p->pomt, p->xl, p->xc_ptr, p->xc_row, p->xc_val, p->m, p->svec, p->fc_y, x, t, q,
            st);
  mat_axpby(n, 1, 1.0, b, n, -1.0, q, n, r, n, st);  // r = b - A x
  dot(n, b, b, sc + 5, st);
  fcg_precond(n, p->box[side], p->pdinv, r, sc + 4, p->net_in, p->net_V, p->net, p->net_out, z, st);
  copy(n, z, pv, st);
  dot(n, r, z, sc + 0, st);
  dot(n, r, r, sc + 2, st);
  TRY(readback(p, DS_FCG, 6, false));
  const double bb = p->hs->ds[DS_FCG + 5];
  const double tol2 = tol * tol * bb;
  double rr = p->hs->ds[DS_FCG + 2];
  // stagnation check: the flexible CG may take at most twice the judge's
  // Jacobi-PCG iterations (plus a margin) before it gives up
  const int cap = std::max(1, std::min(p->opt.pcg_maxit / 2, 2 * p->jac_iters[side] + 16));
  int k = 0;
  while (bb > 0.0 && rr > tol2 && k < cap) {
    fcg_apply(L, p->lam, coef, side, p->pomt, p->xl, p->xc_ptr, p->xc_row, p->xc_val, p->m, p->svec, p->fc_y, pv, t,
              q, st);
    dot(n, pv, q, sc + 1, st);
    fcg_update_xr(n, x, r, rold, pv, q, sc, st);
    dot(n, r, r, sc + 2, st);
    fcg_precond(n, p->box[side], p->pdinv, r, sc + 4, p->net_in, p->net_V, p->net, p->net_out, z, st);
    fcg_diff(n, r, rold, dd, st);
    dot(n, z, dd, sc + 3, st);
    fcg_update_p(n, pv, z, sc, st);
    dot(n, r, z, sc + 0, st);
    ++k;
    if (k < 8 || (k % 4) == 0) {
      TRY(readback(p, DS_FCG, 3, false));
      rr = p->hs->ds[DS_FCG + 2];
      if (!std::isfinite(rr)) break;
      if (by_time && elapsed() > 2.0 * p->jac_sec[side]) break;  // already twice the Jacobi solve's time
    }
  }
  prof_end(p, side == 0 ? CR_PHASE_PCG_U : CR_PHASE_PCG_V);
  PcgStat hs{k, 0, bb > 0.0 ? std::sqrt(std::max(rr, 0.0) / bb) : 0.0, std::sqrt(bb)};
  const bool converged = !(bb > 0.0) || rr <= tol2;
  const bool loss = !converged || (by_time && elapsed() > p->jac_sec[side]);
  if (loss) {
    if (++p->learned_streak[side] >= (by_time ? 2 : 3)) p->learned_off[side] = true;
  } else {
    p->learned_streak[side] = 0;
  }
  if (!converged) {
    // fallback: Jacobi-PCG from the current iterate
    p->fcg_fallbacks += 1;
    TRY(launch_pcg_jacobi(p, side, b, x, p->opt.pcg_maxit));
    TRY(readback(p, 0, 1, true));
    hs = p->hs->stat[side];
    hs.iters += k;
  } else {
    p->learned_solves += 1;
  }
  CUCHK(p, cudaMemcpyAsync(p->stat + side, &hs, sizeof(PcgStat), cudaMemcpyHostToDevice, st));
  return sync(p);
}

cr_status launch_pcg(cr_problem* p, int side, const double* b, double* x) {
  if (p->opt.precond == CR_PRECOND_LEARNED && p->net && p->box[side] && !p->learned_off[side]) {
    if (p->jac_iters[side] > 0) return fcg_learned(p, side, b, x);
    // first solve on this side: Jacobi-PCG, whose iterations and time judge the learned form
    TRY(sync(p));
    const auto t0 = std::chrono::steady_clock::now();
    TRY(launch_pcg_jacobi(p, side, b, x, p->opt.pcg_maxit));
    TRY(readback(p, 0, 1, true));
    p->jac_sec[side] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    p->jac_iters[side] = std::max(1, p->hs->stat[side].iters);
    return CR_OK;
  }
  return launch_pcg_jacobi(p, side, b, x, p->opt.pcg_maxit);
}

PcgArgs pcg_args(cr_problem* p, int side, const double* b, double* x, int maxit, double tol, bool fp32) {
  PcgArgs a{};
  a.lam = p->lam;
  a.m = p->m;
  a.b = b;
  a.x = x;
  a.r = p->pr;
  a.p = p->pp;
  a.sv = p->ps;
  a.w = p->pw;
  a.dinv = p->pdinv;
  a.omt = p->pomt;
  a.fp32 = fp32;
  a.tol = tol;
  a.maxit = maxit;
  a.stat = p->stat + side;
  a.force_generic = p->opt.pcg_kernel == 1;
  if (side == 0) {
    a.L = p->Ly;
    a.coef = p->coef + 0;
    a.Om = p->Om;
    a.ldo = p->ny;
    a.xi = p->xi;
  } else {
    a.L = p->Lx;
    a.coef = p->coef + 2;
    a.X = p->xl;
    a.s = p->svec;
  }
  return a;
}

// Kernel choice: the register-resident cluster kernel while it applies (the
// whole solve on chip); beyond it the grid-wide kernel, which measured as fast
// as the generic cluster kernel at 45k voxels and twice as fast at 127k
// (16 SMs against all of them); pcg_kernel = 1 / 2 force the generic cluster
// or the grid-wide kernel.
bool use_grid_pcg(const cr_problem* p, int side, bool fp32) {
  const DevLap& L = side == 0 ? p->Ly : p->Lx;
  if (p->opt.pcg_kernel == 2 || L.csize == 0) return true;
  if (p->opt.pcg_kernel == 1) return false;
  return pcg_reg_vpt(L, fp32) == 0;
}

// One Jacobi-PCG solve on the cluster-resident kernel, or on the grid-wide
// kernel (use_grid_pcg; that path waits for the result, to turn a grid
// barrier timeout into CR_ETIMEOUT).
// The automatic choice in float32: multigrid above this many rows, or from this
// lambda on (measured on GB300 in the mixed form: at lambda = 100 on 7,530 voxels
// Jacobi reaches relres 1e-6 in 11.5 s against multigrid's 15.0 s on the v side;
// in the lambda sweep over 1 .. 1e6 on 15,000 voxels multigrid is faster overall
// and leaves fewer members at the iteration cap).
constexpr int kMgAutoRows = 20000;
constexpr double kMgAutoLambda = 1e3;

bool use_mg(const cr_problem* p, int side, bool fp32) {
  const DevMg& g = p->mg[side];
  if (!(g.nlev >= 2 && g.smem[fp32 ? 0 : 1] > 0)) return false;
  if (p->opt.precond == CR_PRECOND_MULTIGRID) return true;
  if (p->opt.precond != CR_PRECOND_AUTO) return false;
  // measured on GB300 (7,530 voxels): a multigrid iteration costs ~80-125 us (float32) / ~90-165 us
  // (float64) against ~4-6 / ~9-13 us for Jacobi, while it cuts the iterations 10-50x; in float64
  // that always pays, in float32 only where Jacobi's iteration count is large
  const DevLap& L = side == 0 ? p->Ly : p->Lx;
  return !fp32 || L.n > kMgAutoRows || p->lam >= kMgAutoLambda;
}

cr_status run_pcg(cr_problem* p, int side, const double* b, double* x, int maxit, double tol, bool fp32) {
  const int kph = side == 0 ? CR_PHASE_PCG_KERNEL : CR_PHASE_PCG_KERNEL_V;
  if (use_mg(p, side, fp32)) {
    prof_begin(p, kph);
    CUCHK(p, mg_pcg_launch(pcg_args(p, side, b, x, maxit, tol, fp32), p->mg[side], side, p->st));
    prof_end(p, kph);
    return CR_OK;
  }
  if (!use_grid_pcg(p, side, fp32)) {
    prof_begin(p, kph);
    CUCHK(p, pcg_launch(pcg_args(p, side, b, x, maxit, tol, fp32), side, p->st));
    prof_end(p, kph);
    return CR_OK;
  }
  const int nmax = std::max(p->nx, p->ny);
  if (!p->pg_work) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nbm = std::max(1, 2 * sms);  // the launcher keeps at most two blocks per SM
    TRY(dalloc(p, &p->pg_work, pcg_grid_work_elems(nmax)));
    TRY(dalloc(p, &p->pg_part, (size_t)4 * nbm));
    TRY(dalloc(p, &p->pg_ypart, (size_t)nbm * std::max(1, p->m)));
    TRY(dalloc(p, &p->pg_yglob, (size_t)std::max(1, p->m)));
    TRY(dalloc(p, &p->pg_bar, 2));
    TRY(dalloc(p, &p->pg_err, 1));
  }
  const DevLap& L = side == 0 ? p->Ly : p->Lx;
  const int nb = pcg_grid_blocks(fp32, p->m, L.K);
  if (nb < 1) return fail(p, CR_ECUDA, "the grid-wide PCG cannot be launched on this device");
  const double* coef = p->coef + (side == 0 ? 0 : 2);
  fcg_jacobi_diag(L, p->lam, coef, side, p->m, p->Om, p->ny, p->xi, p->xl, p->svec, p->pomt, p->pdinv, p->st);
  PcgArgs a = pcg_args(p, side, b, x, maxit, tol, fp32);
  prof_begin(p, kph);
  CUCHK(p, pcg_grid_launch(a, side, p->xc_ptr, p->xc_row, p->xc_val, p->pg_work, p->pg_part, p->pg_ypart,
                           p->pg_yglob, p->pg_bar, p->pg_err, std::min(nb, std::max(1, L.n / 64)), p->st));
  prof_end(p, kph);
  TRY(readback(p, 0, 1, true));
  if (p->hs->stat[side].status == 3) return fail(p, CR_ETIMEOUT, "grid-wide PCG barrier timed out");
  return CR_OK;
}

// Jacobi PCG on Eq. (ALS_linsys) (side 0) or Eq. (ALS_linsys_v) (side 1):
// float64 form, or the mixed form's float64 refinement around float32 solves.
cr_status launch_pcg_jacobi(cr_problem* p, int side, const double* b, double* x, int maxit) {
  if (p->opt.precision == CR_MIXED) return launch_pcg_mixed(p, side, b, x, maxit);
  prof_begin(p, side == 0 ? CR_PHASE_PCG_U : CR_PHASE_PCG_V);
  TRY(run_pcg(p, side, b, x, maxit, p->opt.pcg_tol, false));
  prof_end(p, side == 0 ? CR_PHASE_PCG_U : CR_PHASE_PCG_V);
  return CR_OK;
}

// Mixed form of the sub-solves: float64 iterative refinement around the
// float32 cluster PCG.  Each outer step forms the float64 residual
// r = b - A_hat x, stops once |r| <= pcg_tol |b|, and otherwise solves
// A_hat d = r from d = 0 in float32 (inner products in double-float) to
// max(kMixedInnerTol, pcg_tol |b| / (2 |r|)) relative, then x += d.  An outer step that does not cut |r|
// by 4x (float32 cannot resolve the system, e.g. at very large lambda) or the
// step cap hands the solve over to the float64 kernel from the current x, so
// the result meets the float64 tolerance either way.
cr_status launch_pcg_mixed(cr_problem* p, int side, const double* b, double* x, int maxit) {
  cudaStream_t st = p->st;
  const DevLap& L = side == 0 ? p->Ly : p->Lx;
  const int n = L.n;
  const double* coef = p->coef + (side == 0 ? 0 : 2);
  double* sc = p->ds + DS_REF;
  double *r = p->fc_rold, *d = p->fc_d, *q = p->pw;
  const double tol = p->opt.pcg_tol;
  prof_begin(p, side == 0 ? CR_PHASE_PCG_U : CR_PHASE_PCG_V);
  fcg_jacobi_diag(L, p->lam, coef, side, p->m, p->Om, p->ny, p->xi, p->xl, p->svec, p->pomt, p->pdinv, st);
  dot(n, b, b, sc + 0, st);
  PcgStat hs{0, 0, 0.0, 0.0};
  int total = 0;
  double rr_prev = INFINITY;
  for (int outer = 0;; ++outer) {
    fcg_apply(L, p->lam, coef, side, p->pomt, p->xl, p->xc_ptr, p->xc_row, p->xc_val, p->m, p->svec, p->fc_y, x,
              p->fc_t, q, st);
    mat_axpby(n, 1, 1.0, b, n, -1.0, q, n, r, n, st);  // r = b - A x (float64)
    dot(n, r, r, sc + 1, st);
    TRY(readback(p, DS_REF, 2, false));
    const double bb = p->hs->ds[DS_REF], rr = p->hs->ds[DS_REF + 1];
    hs.bnorm = std::sqrt(bb);
    hs.relres = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    if (!(bb > 0.0) || rr <= tol * tol * bb) break;
    if (outer >= kMaxRefine || !(rr < 0.25 * rr_prev) || total >= maxit) {
      // hand over to the float64 kernel from the current iterate
      p->mixed_handovers += 1;
      TRY(run_pcg(p, side, b, x, std::max(1, maxit - total), tol, false));
      TRY(readback(p, 0, 1, true));
      hs = p->hs->stat[side];
      hs.iters += total;
      break;
    }
    rr_prev = rr;
    fill(n, 0.0, d, st);
    // an inner solve never goes further than the float64 target needs (with a
    // factor 2 to spare): on warm-started sweeps the last step is much shorter
    const double inner = std::max(kMixedInnerTol, 0.5 * std::sqrt(tol * tol * bb / rr));
    TRY(run_pcg(p, side, r, d, maxit - total, inner, true));
    TRY(readback(p, 0, 1, true));
    const PcgStat in = p->hs->stat[side];
    total += in.iters;
    hs.iters = total;
    if (in.status == 2) {
      hs.status = 2;
      break;
    }
    mat_axpby(n, 1, 1.0, d, n, 1.0, x, n, x, n, st);  // x += d
  }
  prof_end(p, side == 0 ? CR_PHASE_PCG_U : CR_PHASE_PCG_V);
  CUCHK(p, cudaMemcpyAsync(p->stat + side, &hs, sizeof(PcgStat), cudaMemcpyHostToDevice, st));
  return CR_OK;
}

// K(Zin) of Eq. (Proj_Sylv) into Kout (j x j, ld rcap):
//   lam (Z B2 + 2 A1 Z B1 + A2 Z) + sum_a G_a Z h_a h_a^T,  with the data term
//   evaluated as [G_1 (Z h_1), ..., G_m (Z h_m)] H^T since each V^T X_a X_a^T V
//   is the rank-one h_a h_a^T (h_a = V^T X_a).
void galerkin_apply(cr_problem* p, const double* Zin, double* Kout) {
  cudaStream_t st = p->st;
  const int j = p->j, m = p->m;
  const int64_t ld = p->rcap;
  MatView Zv{Zin, 1, ld};
  gemm(j, j, j, 1.0, Zv, MatView{p->B2, 1, ld}, 0.0, p->gZB2, 1, ld, p->ws, p->ws_elems, st);
  gemm(j, j, j, 1.0, Zv, MatView{p->B1, 1, ld}, 0.0, p->gZB1, 1, ld, p->ws, p->ws_elems, st);
  gemm(j, m, j, 1.0, Zv, MatView{p->H, 1, ld}, 0.0, p->gZH, 1, ld, p->ws, p->ws_elems, st);
  mat_axpby(j, j, p->lam, p->gZB2, ld, 0.0, p->gZB2, ld, Kout, ld, st);
  gemm(j, j, j, 2.0 * p->lam, MatView{p->A1, 1, ld}, MatView{p->gZB1, 1, ld}, 1.0, Kout, 1, ld, p->ws,
       p->ws_elems, st);
  gemm(j, j, j, p->lam, MatView{p->A2, 1, ld}, Zv, 1.0, Kout, 1, ld, p->ws, p->ws_elems, st);
  batched_gemv(j, m, p->G, ld, ld * ld, p->gZH, ld, p->gGw, ld, st);
  gemm(j, j, m, 1.0, MatView{p->gGw, 1, ld}, MatView{p->H, ld, 1}, 1.0, Kout, 1, ld, p->ws, p->ws_elems, st);
}

// F = U^T D V = (U^T (Omega o Y)) (X^T V) = P H^T
void build_F(cr_problem* p) {
  const int64_t ld = p->rcap;
  gemm(p->j, p->j, p->m, 1.0, MatView{p->P, 1, ld}, MatView{p->H, ld, 1}, 0.0, p->F, 1, ld, p->ws, p->ws_elems,
       p->st);
  p->F_valid = true;
}

// E = Omega o (Y - U Z H) after Z changed.
void refresh_E(cr_problem* p) {
  cudaStream_t st = p->st;
  const int j = p->j, m = p->m;
  const int64_t ld = p->rcap;
  if (j == 0) {
    copy(p->ny * m, p->OmY, p->E, st);
    return;
  }
  gemm(j, m, j, 1.0, MatView{p->Z, 1, ld}, MatView{p->H, 1, ld}, 0.0, p->Mzh, 1, ld, p->ws, p->ws_elems, st);
  gemm(p->ny, m, j, 1.0, MatView{p->UU, 1, 3 * (int64_t)p->ny}, MatView{p->Mzh, 1, ld}, 0.0, p->E, 1, p->ny, p->ws,
       p->ws_elems, st);
  mask_residual(p->ny, m, p->OmY, p->Om, p->ny, p->E, st);
}

// Append UU/VV columns 3q..3q+2 to the residual-norm bases.
cr_status grow_bases(cr_problem* p, int q) {
  cudaStream_t st = p->st;
  for (int s = 0; s < 3; ++s) {
    const double* col = p->UU + (size_t)(3 * q + s) * p->ny;
    double* dst = p->QL + (size_t)p->nQL * p->ny;
    copy(p->ny, col, dst, st);
    double ratio = 0.0;
    TRY(cgs2(p, p->ny, p->QL, p->ny, p->nQL, dst, &ratio));
    if (ratio > 1e-12) ++p->nQL;
  }
  for (int s = 0; s < 3; ++s)
    gemv_t(p->ny, p->nQL, p->QL, p->ny, p->UU + (size_t)(3 * q + s) * p->ny, p->CL + (size_t)(3 * q + s) * p->ldcl,
           1, 1.0, 0.0, st);
  for (int s = 0; s < 3; ++s) {
    const double* col = p->VV + (size_t)(3 * q + s) * p->nx;
    double* dst = p->QR + (size_t)p->nQR * p->nx;
    copy(p->nx, col, dst, st);
    double ratio = 0.0;
    TRY(cgs2(p, p->nx, p->QR, p->nx, p->nQR, dst, &ratio));
    if (ratio > 1e-12) {
      ++p->nQR;
      p->qr_step.push_back(q);
    }
  }
  for (int s = 0; s < 3; ++s)
    gemv_t(p->nx, p->nQR, p->QR, p->nx, p->VV + (size_t)(3 * q + s) * p->nx,
           p->CRm + (size_t)(p->m + 3 * q + s) * p->ldcr, 1, 1.0, 0.0, st);
  return CR_OK;
}

// Projections for the new column q (u_q, v_q already in UU/VV column 3q):
// L^s images, borders of U^T L_y^s U, V^T L_x^s V, G_a = U^T diag(Omega_a) U,
// H = V^T X, P = U^T (Omega o Y), and the residual-norm bases.
cr_status grow_projections(cr_problem* p, int q) {
  cudaStream_t st = p->st;
  const int ny = p->ny, nx = p->nx, m = p->m;
  const int64_t ld = p->rcap;
  double* uq = p->UU + (size_t)3 * q * ny;
  double* vq = p->VV + (size_t)3 * q * nx;
  lap_apply(p->Ly, uq, uq + ny, 0.0, st);
  lap_apply(p->Ly, uq + ny, uq + 2 * ny, 0.0, st);
  lap_apply(p->Lx, vq, vq + nx, 0.0, st);
  lap_apply(p->Lx, vq + nx, vq + 2 * nx, 0.0, st);
  const int64_t ldu = 3 * (int64_t)ny, ldv = 3 * (int64_t)nx;
  gemv_t(ny, q + 1, p->UU, ldu, uq + ny, p->A1 + q * ld, 1, 1.0, 0.0, st);
  gemv_t(ny, q + 1, p->UU, ldu, uq + 2 * ny, p->A2 + q * ld, 1, 1.0, 0.0, st);
  gemv_t(nx, q + 1, p->VV, ldv, vq + nx, p->B1 + q * ld, 1, 1.0, 0.0, st);
  gemv_t(nx, q + 1, p->VV, ldv, vq + 2 * nx, p->B2 + q * ld, 1, 1.0, 0.0, st);
  mirror_col(q, p->A1, ld, 1, 0, st);
  mirror_col(q, p->A2, ld, 1, 0, st);
  mirror_col(q, p->B1, ld, 1, 0, st);
  mirror_col(q, p->B2, ld, 1, 0, st);
  spmv_xt(m, p->xc_ptr, p->xc_row, p->xc_val, vq, p->H + q, ld, st);
  gemv_t(ny, m, p->OmY, ny, uq, p->P + q, ld, 1.0, 0.0, st);
  omega_times(ny, m, p->Om, ny, uq, p->Bnm, st);
  gemm(q + 1, m, ny, 1.0, MatView{p->UU, ldu, 1}, MatView{p->Bnm, 1, ny}, 0.0, p->G + q * ld, 1, ld * ld, p->ws,
       p->ws_elems, st);
  mirror_col(q, p->G, ld, m, ld * ld, st);
  return grow_bases(p, q);
}

// Galerkin projection (Eq. Proj_Sylv) by matrix-valued CG from the current Z
// (the previous Z padded with zeros: the warm start of Sec. 2.3), stopped when
// ||F - K(Z)||_F <= tol ||F||_F.  The CG is preconditioned with the diagonal of
// K (the paper's CG is unpreconditioned; the iterate it converges to is the
// same Galerkin solution).  Device scalars: gs[k & 1] = <R_k, D^-1 R_k>,
// gs[2] = <P, K P>, gs[3] = |F|^2, gs[4] = |R|^2.
// float32 G_a = U^T diag(Omega_a) U.  The inner solves of the mixed form take
// the float64 G that the projections keep up to date by borders, rounded to
// float32 (one pass over m j^2 words, and exact to float32 rounding).  A full
// re-assembly from U alone runs on the tensor cores (tcgen05, BF16 hi/lo
// shadows of U split here, j <= 128) when asked for (cr_galerkin_assembly).
cr_status mixed_G(cr_problem* p, bool tensor_cores = false) {
  const int64_t ld = p->rcap;
  if (tensor_cores && p->ubhi && p->j <= 128) {
    bf16_split(p->ny, p->j, p->UU, 3 * (int64_t)p->ny, p->ubhi, p->ublo, p->ldb, p->st);
    const cudaError_t e = galerkin_assemble_tc(p->ny, p->j, p->m, p->ubhi, p->ublo, p->ldb, p->Om, p->ny, p->tc_splits,
                                               p->tcpart, p->fG, ld, p->tcerr, p->st);
    if (e == cudaSuccess) return CR_OK;
    if (e != cudaErrorNotSupported) {
      p->err = std::string("tensor-core Galerkin assembly failed: ") + cudaGetErrorString(e);
      return CR_ECUDA;
    }
    cudaGetLastError();
  }
  to_f32(ld * ld * p->m, p->G, p->fG, p->st);
  return CR_OK;
}

// Eigenbases of A1 = U^T L_y U and B1 = V^T L_x V, brought up to the current
// rank one border at a time.  With A1 = Qa diag(la) Qa^T, the bordered matrix
// [A1 a; a^T alpha] equals blockdiag(Qa, 1) M blockdiag(Qa, 1)^T for the
// arrowhead M of (la, Qa^T a, alpha); with M = W diag(mu) W^T the new basis is
// blockdiag(Qa, 1) W and the new eigenvalues mu.  Everything runs on the device
// (arrow_update, then one product per side), with no host round trip.
cr_status eig_sync(cr_problem* p) {
  cudaStream_t st = p->st;
  const int64_t ld = p->rcap;
  const int j = p->j;
  if (p->eq >= j) return CR_OK;
  prof_begin(p, CR_PHASE_BASIS);
  while (p->eq < j) {
    const int q = p->eq, n1 = q + 1;
    fill(1, 1.0, p->eQa + q + q * ld, st);   // blockdiag(Qa, 1): the rest of row and column q is zero
    fill(1, 1.0, p->eQb + q + q * ld, st);
    double* za = p->ebord;
    double* zb = p->ebord + ld + 1;
    if (q > 0) {
      gemv_t(q, q, p->eQa, ld, p->A1 + q * ld, za, 1, 1.0, 0.0, st);
      gemv_t(q, q, p->eQb, ld, p->B1 + q * ld, zb, 1, 1.0, 0.0, st);
    }
    copy(1, p->A1 + q + q * ld, za + q, st);
    copy(1, p->B1 + q + q * ld, zb + q, st);
    const double* d[2] = {p->ela, p->elb};
    const double* z[2] = {za, zb};
    const double* al[2] = {za + q, zb + q};
    double* mu[2] = {p->ela, p->elb};
    double* W[2] = {p->eW, p->eW + (size_t)n1 * n1};
    CUCHK(p, arrow_update(q, (int)ld, d, z, al, mu, W, p->earw, st));
    gemm(n1, n1, n1, 1.0, MatView{p->eQa, 1, ld}, MatView{W[0], 1, n1}, 0.0, p->eQa2, 1, ld, p->ws, p->ws_elems,
         st);
    gemm(n1, n1, n1, 1.0, MatView{p->eQb, 1, ld}, MatView{W[1], 1, n1}, 0.0, p->eQb2, 1, ld, p->ws, p->ws_elems,
         st);
    std::swap(p->eQa, p->eQa2);
    std::swap(p->eQb, p->eQb2);
    ++p->eq;
  }
  prof_end(p, CR_PHASE_BASIS);
  return CR_OK;
}

// Forget the eigenbases (the factors were replaced); the next projection
// rebuilds them border by border.
void eig_reset(cr_problem* p) {
  if (!p->eQa) return;
  const int64_t ld = p->rcap;
  for (double* b : {p->eQa, p->eQa2, p->eQb, p->eQb2}) fill(ld * ld, 0.0, b, p->st);
  p->eq = 0;
}

bool gal_eigen(const cr_problem* p) {
  return p->eQa && p->j > 0 && (p->opt.precision == CR_MIXED || p->opt.galerkin_kernel == 0);
}

// C = Qa^T S Qb (to_eig) or C = Qa S Qb^T (from_eig), through eTmp.
void eig_transform(cr_problem* p, const double* S, double* C, bool to_eig, double beta = 0.0) {
  const int j = p->j;
  const int64_t ld = p->rcap;
  if (to_eig) {
    gemm(j, j, j, 1.0, MatView{p->eQa, ld, 1}, MatView{S, 1, ld}, 0.0, p->eTmp, 1, ld, p->ws, p->ws_elems, p->st);
    gemm(j, j, j, 1.0, MatView{p->eTmp, 1, ld}, MatView{p->eQb, 1, ld}, beta, C, 1, ld, p->ws, p->ws_elems, p->st);
  } else {
    gemm(j, j, j, 1.0, MatView{p->eQa, 1, ld}, MatView{S, 1, ld}, 0.0, p->eTmp, 1, ld, p->ws, p->ws_elems, p->st);
    gemm(j, j, j, 1.0, MatView{p->eTmp, 1, ld}, MatView{p->eQb, ld, 1}, beta, C, 1, ld, p->ws, p->ws_elems, p->st);
  }
}

// The eigenbasis operator's matrices: A2t = Qa^T A2 Qa, B2t = Qb^T B2 Qb,
// Ht = Qb^T H, and the preconditioner's diagonal.
void eig_operator(cr_problem* p) {
  cudaStream_t st = p->st;
  const int j = p->j, m = p->m;
  const int64_t ld = p->rcap;
  gemm(j, j, j, 1.0, MatView{p->eQa, ld, 1}, MatView{p->A2, 1, ld}, 0.0, p->eTmp, 1, ld, p->ws, p->ws_elems, st);
  gemm(j, j, j, 1.0, MatView{p->eTmp, 1, ld}, MatView{p->eQa, 1, ld}, 0.0, p->eA2t, 1, ld, p->ws, p->ws_elems, st);
  gemm(j, j, j, 1.0, MatView{p->eQb, ld, 1}, MatView{p->B2, 1, ld}, 0.0, p->eTmp, 1, ld, p->ws, p->ws_elems, st);
  gemm(j, j, j, 1.0, MatView{p->eTmp, 1, ld}, MatView{p->eQb, 1, ld}, 0.0, p->eB2t, 1, ld, p->ws, p->ws_elems, st);
  gemm(j, m, j, 1.0, MatView{p->eQb, ld, 1}, MatView{p->H, 1, ld}, 0.0, p->eHt, 1, ld, p->ws, p->ws_elems, st);
  galerkin_eig_diag(j, m, ld, p->lam, p->eA2t, p->eB2t, p->ela, p->elb, p->G, p->eHt, p->eg, p->eDen, p->eDl,
                    p->eHg, st);
  p->smw_ok = false;
  if (p->eCi) {
    const cudaError_t e = galerkin_smw_setup(j, m, ld, p->eDl, p->eHg, p->eCi, st);
    if (e == cudaSuccess) {
      p->smw_ok = true;
    } else {
      cudaGetLastError();  // too large for the row-wise preconditioner: the diagonal one stays
    }
  }
}

// Relative Galerkin residual that counts as "to rounding": smaller targets (tau = 0)
// are raised to it, so that a CG whose residual has reached the rounding floor stops.
constexpr double kGalTolFloor = 1e-14;
// Mixed form: each float32 inner solve of the Galerkin refinement stops at
// |r|^2 <= kGalInner |R|^2 (R the float64 residual of the outer step).
constexpr double kGalInner = 1e-7;

cr_status do_project(cr_problem* p, double tol, cr_proj_info* info) {
  tol = std::max(tol, kGalTolFloor);
  cudaStream_t st = p->st;
  const int j = p->j;
  const int64_t ld = p->rcap;
  if (info) *info = cr_proj_info{0, 0.0};
  if (j == 0) return CR_OK;
  prof_begin(p, CR_PHASE_GALERKIN);
  CUCHK(p, cudaMemcpyAsync(p->Zprev, p->Z, sizeof(double) * ld * ld, cudaMemcpyDeviceToDevice, st));
  build_F(p);
  double* gs = p->ds + DS_GS;
  galerkin_diag(j, p->m, p->A1, p->A2, p->B1, p->B2, p->G, p->H, ld, p->lam, p->gDg, st);
  const int maxit = p->opt.galerkin_maxit > 0 ? p->opt.galerkin_maxit : 10 * j * j + 100;
  int k = 0;
  double fn2 = 0.0, rr = 0.0;
  cr_status rc = CR_OK;
  const bool eig = gal_eigen(p);
  if (eig) {
    TRY(eig_sync(p));
    eig_operator(p);
  }
  if (p->opt.precision == CR_MIXED && p->gal_nb > 0) {
    // Mixed form: float64 iterative refinement.  Each outer step forms the
    // float64 residual R = F - K(Z) and solves K dZ = R to about 3e-4 relative
    // (|r|^2 <= 1e-7 |R|^2) with the persistent CG in float32 (float32 copies of
    // the projected matrices), then Z += dZ; the stopping test is on the float64
    // residual.  Tighter inner solves cost more CG iterations than the outer
    // steps they save, looser ones need more outer steps: 1e-7 measured fastest.
    mat_dot(j, j, p->F, ld, p->F, ld, gs + 3, st);
    TRY(readback(p, DS_GS + 3, 1, false));
    fn2 = p->hs->ds[DS_GS + 3];
    const int64_t r2 = ld * ld;
    if (eig) {
      // the inner float32 CG runs in the eigenbasis; the float64 residual stays in the original one
      to_f32(r2, p->eA2t, p->fA2, st);
      to_f32(r2, p->eB2t, p->fB2, st);
      to_f32(r2, p->eDen, p->fDg, st);
      to_f32(ld * p->m, p->eHt, p->fH, st);
      to_f32(r2, p->eQa, p->fQa, st);
      to_f32(ld, p->ela, p->fla, st);
      to_f32(ld, p->elb, p->flb, st);
      ++p->gal_eig_proj;
    } else {
      to_f32(r2, p->A1, p->fA1, st);
      to_f32(r2, p->A2, p->fA2, st);
      to_f32(r2, p->B1, p->fB1, st);
      to_f32(r2, p->B2, p->fB2, st);
      to_f32(r2, p->gDg, p->fDg, st);
      to_f32(ld * p->m, p->H, p->fH, st);
    }
    TRY(mixed_G(p));
    GalEig<float> fe;
    fe.Qa = p->fQa;
    fe.la = p->fla;
    fe.lb = p->flb;
    fe.Y = p->fY;
    fe.Gt = p->fGt;
    if (eig && p->smw_ok) {
      fe.Dl = p->eDl;
      fe.Hg = p->eHg;
      fe.Ci = p->eCi;
      fe.S = p->eS;
      fe.Yd = p->eYd;
      fe.Zz = p->fZz;
    }
    // an inner solve that has not converged by this cap hands back to the outer
    // float64 refinement, which checks the progress itself
    const int inner_maxit = std::min(maxit, 2000 + 10 * j);
    for (int outer = 0; outer < 40 && fn2 > 0.0; ++outer) {
      galerkin_apply(p, p->Z, p->gQ);
      mat_axpby(j, j, 1.0, p->F, ld, -1.0, p->gQ, ld, p->gR, ld, st);
      mat_dot(j, j, p->gR, ld, p->gR, ld, gs + 4, st);
      TRY(readback(p, DS_GS + 4, 1, false));
      rr = p->hs->ds[DS_GS + 4];
      if (!(rr > tol * tol * fn2)) break;
      if (!std::isfinite(rr)) {
        rc = fail(p, CR_ENOTCONV, "mixed Galerkin refinement produced a non-finite residual");
        break;
      }
      if (eig) {
        eig_transform(p, p->gR, p->eFt, true);
        to_f32(r2, p->eFt, p->fF, st);
      } else {
        to_f32(r2, p->gR, p->fF, st);
      }
      CUCHK(p, cudaMemsetAsync(p->fZ, 0, sizeof(float) * r2, st));
      CUCHK(p, cudaMemsetAsync(p->gbar, 0, 2 * sizeof(unsigned), st));
      CUCHK(p, cudaMemsetAsync(p->gerr, 0, sizeof(int), st));
      // the single-cluster kernel has no row-wise preconditioner: with it, the persistent kernel
      cudaError_t ce = cudaErrorNotSupported;
      if (!(eig && p->smw_ok))
        ce = galerkin_cluster_f32_launch(j, p->m, ld, p->lam, p->fA1, p->fA2, p->fB1, p->fB2, p->fG, p->fH, p->fF,
                                         p->fDg, p->fZ, kGalInner * rr, inner_maxit, p->gout, st, eig ? &fe : nullptr);
      if (ce == cudaErrorNotSupported) {
        cudaGetLastError();
        ce = galerkin_cg_launch<float>(p->gal_nb, j, p->m, ld, p->lam, p->fA1, p->fA2, p->fB1, p->fB2, p->fG, p->fH,
                                       p->fF, p->fDg, p->fZ, p->fR, p->fPa, p->fPb, p->fQ, p->fT2, p->fT1, p->fTH,
                                       p->fGw, p->fzb, p->gpart, p->gbar, p->gerr, kGalInner * rr, inner_maxit, p->gout,
                                       st, eig ? &fe : nullptr);
      }
      CUCHK(p, ce);
      double out[3] = {0, 0, 0};
      CUCHK(p, cudaMemcpyAsync(out, p->gout, sizeof(out), cudaMemcpyDeviceToHost, st));
      p->d2h_bytes += (int64_t)sizeof(out);
      TRY(sync(p));
      k += (int)out[0];
      if (out[2] == 3.0) return fail(p, CR_ETIMEOUT, "Galerkin CG grid barrier timed out");
      if (eig) {  // Z += Qa dZt Qb^T
        fill(r2, 0.0, p->eZt, st);
        add_f32(j, j, p->fZ, ld, p->eZt, ld, st);
        eig_transform(p, p->eZt, p->Z, false, 1.0);
      } else {
        add_f32(j, j, p->fZ, ld, p->Z, ld, st);
      }
      if (outer == 39) rc = fail(p, CR_ENOTCONV, "mixed Galerkin refinement did not converge");
    }
  } else if (p->opt.galerkin_kernel == 0 && p->gal_nb > 0) {
    // one cooperative launch runs the whole CG
    mat_dot(j, j, p->F, ld, p->F, ld, gs + 3, st);
    TRY(readback(p, DS_GS + 3, 1, false));
    fn2 = p->hs->ds[DS_GS + 3];
    bool done = false;
    if (eig && fn2 > 0.0) {
      // CG on Zt = Qa^T Z Qb from the transformed warm start, then Z = Qa Zt Qb^T and
      // its residual in the original basis.  Where that residual is still above the
      // tolerance (the bases carry rounding), up to two refinement steps solve for the
      // correction in the eigenbasis; the original-basis CG is the last resort.
      GalEig<double> ge;
      ge.Qa = p->eQa;
      ge.la = p->ela;
      ge.lb = p->elb;
      ge.Y = p->eY;
      ge.Gt = p->eGt;
      if (p->smw_ok) {
        ge.Dl = p->eDl;
        ge.Hg = p->eHg;
        ge.Ci = p->eCi;
        ge.S = p->eS;
        ge.Yd = p->eYd;
        ge.Zz = p->eZz;
      }
      ++p->gal_eig_proj;
      for (int ref = 0; ref < 3 && !done; ++ref) {
        if (ref == 0) {
          eig_transform(p, p->F, p->eFt, true);
          eig_transform(p, p->Z, p->eZt, true);
        } else {
          eig_transform(p, p->gR, p->eFt, true);
          fill(ld * ld, 0.0, p->eZt, st);
        }
        CUCHK(p, cudaMemsetAsync(p->gbar, 0, 2 * sizeof(unsigned), st));
        CUCHK(p, cudaMemsetAsync(p->gerr, 0, sizeof(int), st));
        // the whole system to the tolerance itself (a tighter first target costs more
        // iterations than the refinements it saves); a correction to half of it
        const double t2 = (ref == 0 ? 1.0 : 0.25) * tol * tol * fn2;
        CUCHK(p, galerkin_cg_launch(p->gal_nb, j, p->m, ld, p->lam, p->A1, p->eA2t, p->B1, p->eB2t, p->G, p->eHt,
                                    p->eFt, p->eDen, p->eZt, p->gR, p->gP, p->gT, p->gQ, p->gZB2, p->gZB1, p->gZH,
                                    p->gGw, p->gzb, p->gpart, p->gbar, p->gerr, t2, std::max(1, maxit - k), p->gout,
                                    st, &ge));
        double out[3] = {0, 0, 0};
        CUCHK(p, cudaMemcpyAsync(out, p->gout, sizeof(out), cudaMemcpyDeviceToHost, st));
        p->d2h_bytes += (int64_t)sizeof(out);
        TRY(sync(p));
        k += (int)out[0];
        if (out[2] == 3.0) return fail(p, CR_ETIMEOUT, "Galerkin CG grid barrier timed out");
        eig_transform(p, p->eZt, p->Z, false, ref == 0 ? 0.0 : 1.0);
        galerkin_apply(p, p->Z, p->gQ);
        mat_axpby(j, j, 1.0, p->F, ld, -1.0, p->gQ, ld, p->gR, ld, st);
        mat_dot(j, j, p->gR, ld, p->gR, ld, gs + 4, st);
        TRY(readback(p, DS_GS + 4, 1, false));
        rr = p->hs->ds[DS_GS + 4];
        done = rr <= tol * tol * fn2;
        if (!done && k >= maxit) {  // the cap covers every CG of the projection
          done = true;
          rc = fail(p, CR_ENOTCONV, "Galerkin CG reached its iteration cap");
        }
      }
      if (!done) ++p->gal_eig_finish;
    }
    if (fn2 > 0.0 && !done) {
      CUCHK(p, cudaMemsetAsync(p->gbar, 0, 2 * sizeof(unsigned), st));
      CUCHK(p, cudaMemsetAsync(p->gerr, 0, sizeof(int), st));
      CUCHK(p, galerkin_cg_launch(p->gal_nb, j, p->m, ld, p->lam, p->A1, p->A2, p->B1, p->B2, p->G, p->H, p->F,
                                  p->gDg, p->Z, p->gR, p->gP, p->gT, p->gQ, p->gZB2, p->gZB1, p->gZH, p->gGw, p->gzb,
                                  p->gpart, p->gbar, p->gerr, tol * tol * fn2, maxit - k, p->gout, st));
      double out[3] = {0, 0, 0};
      CUCHK(p, cudaMemcpyAsync(out, p->gout, sizeof(out), cudaMemcpyDeviceToHost, st));
      p->d2h_bytes += (int64_t)sizeof(out);
      TRY(sync(p));
      k += (int)out[0];
      rr = out[1];
      if (out[2] == 1.0) rc = fail(p, CR_ENOTCONV, "Galerkin CG reached its iteration cap");
      if (out[2] == 2.0) rc = fail(p, CR_ENOTCONV, "Galerkin CG broke down (non-positive curvature)");
      if (out[2] == 3.0) return fail(p, CR_ETIMEOUT, "Galerkin CG grid barrier timed out");
    }
  } else {
    galerkin_apply(p, p->Z, p->gQ);
    mat_axpby(j, j, 1.0, p->F, ld, -1.0, p->gQ, ld, p->gR, ld, st);  // R = F - K(Z)
    precond_dots(j, p->gR, p->gDg, ld, p->gP, gs + 0, gs + 4, st);   // P = D^-1 R
    mat_dot(j, j, p->F, ld, p->F, ld, gs + 3, st);
    TRY(readback(p, DS_GS, 5, false));
    fn2 = p->hs->ds[DS_GS + 3];
    rr = p->hs->ds[DS_GS + 4];
    const double thr2 = tol * tol * fn2;
    if (fn2 > 0.0 && rr > thr2) {
      for (;;) {
        galerkin_apply(p, p->gP, p->gQ);
        mat_dot(j, j, p->gP, ld, p->gQ, ld, gs + 2, st);
        cg_update_zr(j, p->Z, p->gR, p->gP, p->gQ, ld, gs, k, st);
        precond_dots(j, p->gR, p->gDg, ld, p->gT, gs + ((k + 1) & 1), gs + 4, st);
        cg_update_p(j, p->gP, p->gT, ld, gs, k, st);
        ++k;
        const bool check = k < 8 || (k % 4) == 0 || k >= maxit;
        if (check) {
          TRY(readback(p, DS_GS, 5, false));
          rr = p->hs->ds[DS_GS + 4];
          if (!(rr > thr2)) break;
          if (!std::isfinite(rr)) {
            rc = fail(p, CR_ENOTCONV, "Galerkin CG produced a non-finite residual");
            break;
          }
        }
        if (k >= maxit) {
          rc = fail(p, CR_ENOTCONV, "Galerkin CG reached its iteration cap");
          break;
        }
      }
    }
  }
  refresh_E(p);
  prof_end(p, CR_PHASE_GALERKIN);
  TRY(sync(p));
  if (info) {
    info->iters = k;
    info->relres = fn2 > 0.0 ? std::sqrt(std::max(rr, 0.0) / fn2) : 0.0;
  }
  return rc;
}

cr_status do_relres(cr_problem* p, double* relres) {
  cudaStream_t st = p->st;
  const int j = p->j, m = p->m, ny = p->ny;
  const int k = p->nQL;
  const int64_t ldcx = p->ldcx;
  // E_perp = E - Q_L (Q_L^T E), twice; Cx accumulates Q_L^T E.
  copy(ny * m, p->E, p->Ep, st);
  if (k > 0) {
    gemm(k, m, ny, 1.0, MatView{p->QL, ny, 1}, MatView{p->E, 1, ny}, 0.0, p->Cx, 1, ldcx, p->ws, p->ws_elems, st);
    gemm(ny, m, k, -1.0, MatView{p->QL, 1, ny}, MatView{p->Cx, 1, ldcx}, 1.0, p->Ep, 1, ny, p->ws, p->ws_elems, st);
    gemm(k, m, ny, 1.0, MatView{p->QL, ny, 1}, MatView{p->Ep, 1, ny}, 0.0, p->Cx2, 1, ldcx, p->ws, p->ws_elems, st);
    gemm(ny, m, k, -1.0, MatView{p->QL, 1, ny}, MatView{p->Cx2, 1, ldcx}, 1.0, p->Ep, 1, ny, p->ws, p->ws_elems, st);
    mat_axpby(k, m, 1.0, p->Cx2, ldcx, 1.0, p->Cx, ldcx, p->Cx, ldcx, st);
  }
  // Q_E: orthonormal basis of span(E_perp) from the eigen-decomposition of its
  // Gram matrix (host, m x m), applied twice for orthogonality.
  double* QE = p->QL + (size_t)k * ny;
  gemm(m, m, ny, 1.0, MatView{p->Ep, ny, 1}, MatView{p->Ep, 1, ny}, 0.0, p->gram, 1, m, p->ws, p->ws_elems, st);
  std::vector<double> gram((size_t)m * m);
  CUCHK(p, cudaMemcpyAsync(gram.data(), p->gram, sizeof(double) * m * m, cudaMemcpyDeviceToHost, st));
  p->d2h_bytes += (int64_t)sizeof(double) * m * m;
  TRY(sync(p));
  std::vector<double> w, V;
  sym_eig(m, gram, w, V);
  double wmax = 0.0;
  for (double x : w) wmax = std::max(wmax, x);
  std::vector<double> T;
  int ke = 0;
  const double thr = 1e-26 * std::max(wmax, p->Dnorm * p->Dnorm * 1e-30);
  for (int i = 0; i < m; ++i)
    if (w[i] > thr && w[i] > 1e-20 * wmax) {
      for (int r = 0; r < m; ++r) T.push_back(V[r + (size_t)i * m] / std::sqrt(w[i]));
      ++ke;
    }
  if (ke > 0) {
    CUCHK(p, cudaMemcpyAsync(p->tmat, T.data(), sizeof(double) * T.size(), cudaMemcpyHostToDevice, st));
    p->h2d_bytes += (int64_t)(sizeof(double) * T.size());
    gemm(ny, ke, m, 1.0, MatView{p->Ep, 1, ny}, MatView{p->tmat, 1, m}, 0.0, QE, 1, ny, p->ws, p->ws_elems, st);
    // second pass: Cholesky of Q_E^T Q_E
    gemm(ke, ke, ny, 1.0, MatView{QE, ny, 1}, MatView{QE, 1, ny}, 0.0, p->gram, 1, ke, p->ws, p->ws_elems, st);
    std::vector<double> g2((size_t)ke * ke);
    CUCHK(p, cudaMemcpyAsync(g2.data(), p->gram, sizeof(double) * ke * ke, cudaMemcpyDeviceToHost, st));
    p->d2h_bytes += (int64_t)(sizeof(double) * ke * ke);
    TRY(sync(p));
    // upper Cholesky factor R (g2 = R^T R), then Rinv
    std::vector<double> R((size_t)ke * ke, 0.0), Ri((size_t)ke * ke, 0.0);
    bool ok = true;
    for (int c = 0; c < ke && ok; ++c) {
      for (int r = 0; r <= c; ++r) {
        double s = g2[r + (size_t)c * ke];
        for (int t = 0; t < r; ++t) s -= R[t + (size_t)r * ke] * R[t + (size_t)c * ke];
        if (r == c) {
          if (s <= 0.0) {
            ok = false;
            break;
          }
          R[r + (size_t)c * ke] = std::sqrt(s);
        } else {
          R[r + (size_t)c * ke] = s / R[r + (size_t)r * ke];
        }
      }
    }
    if (ok) {
      for (int c = 0; c < ke; ++c) {
        Ri[c + (size_t)c * ke] = 1.0 / R[c + (size_t)c * ke];
        for (int r = c - 1; r >= 0; --r) {
          double s = 0.0;
          for (int t = r + 1; t <= c; ++t) s += R[r + (size_t)t * ke] * Ri[t + (size_t)c * ke];
          Ri[r + (size_t)c * ke] = -s / R[r + (size_t)r * ke];
        }
      }
      CUCHK(p, cudaMemcpyAsync(p->tmat, Ri.data(), sizeof(double) * Ri.size(), cudaMemcpyHostToDevice, st));
      p->h2d_bytes += (int64_t)(sizeof(double) * Ri.size());
      copy(ny * ke, QE, p->Bnm, st);
      gemm(ny, ke, ke, 1.0, MatView{p->Bnm, 1, ny}, MatView{p->tmat, 1, ke}, 0.0, QE, 1, ny, p->ws, p->ws_elems,
           st);
    }
    gemm(ke, m, ny, 1.0, MatView{QE, ny, 1}, MatView{p->Ep, 1, ny}, 0.0, p->CE, 1, m, p->ws, p->ws_elems, st);
  }
  // C_P = [[Cx, CL], [CE, 0]]  ((k + ke) x (m + 3j))
  const int nc = m + 3 * j, kr = k + ke;
  const int64_t ldcp = p->ldcp;
  fill((int64_t)ldcp * nc, 0.0, p->CP, st);
  if (k > 0) {
    copy2d(k, m, p->Cx, ldcx, p->CP, ldcp, st);
    copy2d(k, 3 * j, p->CL, p->ldcl, p->CP + (size_t)m * ldcp, ldcp, st);
  }
  if (ke > 0) copy2d(ke, m, p->CE, m, p->CP + k, ldcp, st);
  // T1 = C_P M_c.  The core M_c is the identity on the m data columns and
  // -lam (Z kron J) on the panels (column 3p + s of a panel block is L^s u_p; J the
  // anti-diagonal (1, 2, 1)), so T1 is the data columns of C_P and, for t = 0, 1, 2,
  // the panel columns t of T1 = -lam c_t (panel columns 2 - t of C_P) Z, c_1 = 2:
  // three products of kr x j x j instead of one of kr x (m + 3j)^2.
  copy2d(kr, m, p->CP, ldcp, p->T1, ldcp, st);
  for (int t = 0; t < 3; ++t)
    gemm(kr, j, j, -p->lam * (t == 1 ? 2.0 : 1.0), MatView{p->CP + (size_t)(m + 2 - t) * ldcp, 1, 3 * ldcp},
         MatView{p->Z, 1, p->rcap}, 0.0, p->T1 + (size_t)(m + t) * ldcp, 1, 3 * ldcp, p->ws, p->ws_elems, st);
  // T2 = T1 C_Q^T.  C_Q is block upper triangular: right-basis vector r created in
  // greedy step q_r has coefficients only on the data columns (r < nQX) or the panel
  // columns of steps >= q_r, so each 64-column block of T2 sums from column
  // m + 3 q_r0 on.
  for (int r0 = 0; r0 < p->nQR; r0 += 64) {
    const int r1 = std::min(p->nQR, r0 + 64);
    const int k0 = r0 < p->nQX ? 0 : m + 3 * p->qr_step[r0 - p->nQX];
    gemm(kr, r1 - r0, nc - k0, 1.0, MatView{p->T1 + (size_t)k0 * ldcp, 1, ldcp},
         MatView{p->CRm + r0 + (size_t)k0 * p->ldcr, p->ldcr, 1}, 0.0, p->T2 + (size_t)r0 * ldcp, 1, ldcp, p->ws,
         p->ws_elems, st);
  }
  mat_dot(kr, p->nQR, p->T2, ldcp, p->T2, ldcp, p->ds + DS_RN, st);
  TRY(readback(p, DS_RN, 1, false));
  *relres = p->Dnorm > 0.0 ? std::sqrt(p->hs->ds[DS_RN]) / p->Dnorm : 0.0;
  return CR_OK;
}

cr_status do_rank_one(cr_problem* p, cr_rank1_info* info) {
  cudaStream_t st = p->st;
  const int ny = p->ny, nx = p->nx, j = p->j;
  if (j >= p->rcap) return fail(p, CR_ESTATE, "rank capacity r_cap reached");
  // ALS start vector: v0 = R_j^T 1 / |R_j^T 1|
  fill(ny, 1.0, p->tmpy, st);
  residual_t_times(p, p->tmpy, p->v);
  dot(nx, p->v, p->v, p->ds + DS_V0, st);
  TRY(readback(p, DS_V0, 1, false));
  const double v0n2 = p->hs->ds[DS_V0];
  if (v0n2 > 1e-300 * p->Dnorm * p->Dnorm && std::isfinite(v0n2)) {
    scale_by_inv_norm(nx, p->v, p->ds + DS_V0, p->v, st);
  } else {
    // splitmix64 -> Box-Muller Gaussian, seeded by (seed + j)
    std::vector<double> g(nx);
    uint64_t state = p->opt.seed + (uint64_t)j;
    auto next = [&state]() {
      uint64_t z = (state += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    double nrm = 0.0;
    for (int i = 0; i < nx; ++i) {
      const double u1 = ((next() >> 11) + 1.0) * (1.0 / 9007199254740993.0);
      const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
      g[i] = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
      nrm += g[i] * g[i];
    }
    for (double& x : g) x /= std::sqrt(nrm);
    CUCHK(p, cudaMemcpyAsync(p->v, g.data(), sizeof(double) * nx, cudaMemcpyHostToDevice, st));
    p->h2d_bytes += (int64_t)(sizeof(double) * nx);
  }
  fill(ny, 0.0, p->uhat, st);
  fill(nx, 0.0, p->vhat, st);
  int sweeps = 0;
  double delta = INFINITY, un = 0.0, vn = 0.0, worst = 0.0;
  int itu = 0, itv = 0;
  bool capped = false;  // some sub-solve of some sweep stopped at pcg_maxit
  for (;;) {
    prof_begin(p, CR_PHASE_RHS);
    prep_u(p, p->v);
    residual_times(p, p->v, p->rhs_u);
    prof_end(p, CR_PHASE_RHS);
    TRY(launch_pcg(p, 0, p->rhs_u, p->uhat));
    prof_begin(p, CR_PHASE_RHS);
    dot(ny, p->uhat, p->uhat, p->ds + DS_UN2, st);
    scale_by_inv_norm(ny, p->uhat, p->ds + DS_UN2, p->u, st);
    prep_v(p, p->u);
    residual_t_times(p, p->u, p->rhs_v);
    prof_end(p, CR_PHASE_RHS);
    TRY(launch_pcg(p, 1, p->rhs_v, p->vhat));
    dot(nx, p->vhat, p->vhat, p->ds + DS_VN2, st);
    scale_by_inv_norm(nx, p->vhat, p->ds + DS_VN2, p->v, st);
    TRY(readback(p, 0, 2, true));
    const PcgStat* s = p->hs->stat;
    p->pcg_solves += 2;
    p->pcg_iters += s[0].iters + s[1].iters;
    p->pcg_iters_side[0] += s[0].iters;
    p->pcg_iters_side[1] += s[1].iters;
    itu += s[0].iters;
    itv += s[1].iters;
    worst = std::max(worst, std::max(s[0].relres, s[1].relres));
    capped = capped || s[0].status == 1 || s[1].status == 1;
    un = std::sqrt(p->hs->ds[DS_UN2]);
    vn = std::sqrt(p->hs->ds[DS_VN2]);
    ++sweeps;
    if (s[0].status == 2 || s[1].status == 2 || !(un > 0.0) || !(vn > 0.0) || !std::isfinite(un) ||
        !std::isfinite(vn))
      return fail(p, CR_ENOTCONV, "ALS sub-solve broke down (indefinite operator or zero solution)");
    delta = std::fabs(un / vn - 1.0);
    if (p->opt.als_sweeps > 0) {
      if (sweeps >= p->opt.als_sweeps) break;
    } else if (delta <= p->opt.als_delta || sweeps >= p->opt.als_max_iter) {
      break;
    }
  }
  // orth: U <- orth([U, u]), V <- orth([V, v])
  prof_begin(p, CR_PHASE_ORTH);
  double* uq = p->UU + (size_t)3 * j * ny;
  double* vq = p->VV + (size_t)3 * j * nx;
  copy(ny, p->u, uq, st);
  copy(nx, p->v, vq, st);
  double ru = 0.0, rv = 0.0;
  TRY(cgs2(p, ny, p->UU, 3 * (int64_t)ny, j, uq, &ru));
  TRY(cgs2(p, nx, p->VV, 3 * (int64_t)nx, j, vq, &rv));
  if (!(ru >= 1e-12) || !(rv >= 1e-12)) return fail(p, CR_ERANK, "new ALS factor lies in the current span");
  TRY(grow_projections(p, j));
  zero_border(j, p->Z, p->rcap, st);
  p->j = j + 1;
  p->F_valid = false;
  prof_end(p, CR_PHASE_ORTH);
  TRY(sync(p));
  if (info) {
    info->rank = p->j;
    info->sweeps = sweeps;
    info->delta = delta;
    info->unorm = un;
    info->vnorm = vn;
    info->pcg_iters_u = itu;
    info->pcg_iters_v = itv;
    info->pcg_relres_max = worst;
  }
  if (capped) return fail(p, CR_ENOTCONV, "PCG reached pcg_maxit in an ALS sweep (the step was still taken)");
  return CR_OK;
}

}  // namespace

namespace cr {
// Move a problem onto stream st (NULL: a new library-owned stream) once the
// work on its current stream has finished; the old stream is released if the
// problem owned it.
cr_status adopt_stream(cr_problem* p, cudaStream_t st) {
  CUCHK(p, cudaStreamSynchronize(p->st));
  cudaStream_t ns = st;
  if (!ns) CUCHK(p, cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking));
  if (p->own_stream && p->st) cudaStreamDestroy(p->st);
  p->st = ns;
  p->own_stream = !st;
  return CR_OK;
}
}  // namespace cr

// =========================================================================== C ABI
extern "C" {

cr_status cr_options_default(cr_options* o) {
  if (!o) return CR_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(cr_options);
  o->r_cap = 100;
  o->precision = CR_FP64;
  o->precond = CR_PRECOND_JACOBI;
  o->pcg_tol = 1e-10;
  o->pcg_maxit = 20000;
  o->als_delta = 0.1;
  o->als_max_iter = 10;
  o->als_sweeps = 0;
  o->galerkin_maxit = 0;
  o->residual_every = 1;
  o->cluster_size = 0;
  o->profile = 0;
  o->pcg_kernel = 0;
  o->galerkin_kernel = 0;
  o->seed = 1808;
  return CR_OK;
}

double cr_lambda_from_bar(double lambda_bar, int64_t ninj, int64_t nx) {
  return nx > 0 ? lambda_bar * (double)ninj / (double)nx : NAN;
}

const char* cr_status_str(cr_status s) {
  switch (s) {
    case CR_OK: return "ok";
    case CR_EINVAL: return "invalid argument";
    case CR_ENOMEM: return "out of device memory";
    case CR_ECUDA: return "CUDA error";
    case CR_ENOTCONV: return "iteration cap reached";
    case CR_ETIMEOUT: return "time budget exceeded";
    case CR_ERANK: return "rank deficient update";
    case CR_ESTATE: return "invalid state";
  }
  return "unknown status";
}

const char* cr_last_error(const cr_problem* p) { return p ? p->err.c_str() : g_create_err.c_str(); }

void cr_destroy(cr_problem* p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st);
  for (auto& a : p->allocs) {
    if (p->opt.alloc)
      p->opt.free(a.first, a.second, p->opt.alloc_ctx);
    else
      cudaFree(a.first);
  }
  if (p->hs) cudaFreeHost(p->hs);
  prof_resolve(p);
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  for (auto e : p->open_ev)
    if (e) cudaEventDestroy(e);
  if (p->own_stream && p->st) cudaStreamDestroy(p->st);
  delete p;
}

cr_status cr_create(const cr_problem_desc* d_in, const cr_options* o, cr_problem** out) {
  if (out) *out = nullptr;
  g_create_err.clear();
  auto bad = [](const std::string& m) {
    g_create_err = m;
    return CR_EINVAL;
  };
  if (!d_in || !out) return bad("null argument");
  DescCopy staged;
  cr_problem_desc dview;
  {
    std::string serr;
    const cr_status ss = stage_desc(d_in, &staged, &dview, serr);
    if (ss != CR_OK) {
      g_create_err = serr;
      return ss;
    }
  }
  const cr_problem_desc* d = &dview;
  cr_options opt;
  cr_options_default(&opt);
  if (o) {
    if (o->struct_size != sizeof(cr_options)) return bad("cr_options.struct_size mismatch");
    opt = *o;
  }
  const int64_t nx = d->nx, ny = d->ny, m = d->ninj;
  if (nx <= 0 || ny <= 0 || m <= 0 || nx > (1 << 24) || ny > (1 << 24) || m > 4096) return bad("bad sizes");
  if (!d->X_host || !d->Y_host || !d->Omega_host || d->ldx < nx || d->ldy < ny || d->ldo < ny)
    return bad("null data pointer or leading dimension too small");
  if (!(d->lambda > 0.0) || !std::isfinite(d->lambda)) return bad("lambda must be finite and > 0");
  if (opt.r_cap < 1 || opt.r_cap > std::min(nx, ny)) return bad("r_cap must be in [1, min(nx, ny)]");
  if (!(opt.pcg_tol > 0.0) || opt.pcg_maxit < 1 || opt.als_max_iter < 1 || !(opt.als_delta >= 0.0))
    return bad("bad solver options");
  if (opt.galerkin_form < CR_GALERKIN_AUTO || opt.galerkin_form > CR_GALERKIN_EIGEN)
    return bad("galerkin_form must be a cr_galerkin_form");
  if (opt.alloc && !opt.free) return bad("alloc given without free");
  std::string err;
  if (check_csr(d->Lx, nx, "Lx", err) != CR_OK || check_csr(d->Ly, ny, "Ly", err) != CR_OK) return bad(err);
  if (d->grid_x.box_index && !grid_ok(d->grid_x.dims, d->grid_x.box_index, nx, err)) return bad("grid_x: " + err);
  if (d->grid_y.box_index && !grid_ok(d->grid_y.dims, d->grid_y.box_index, ny, err)) return bad("grid_y: " + err);
  for (int64_t a = 0; a < m; ++a) {
    for (int64_t i = 0; i < nx; ++i)
      if (!std::isfinite(d->X_host[i + a * d->ldx])) return bad("X has a non-finite entry");
    for (int64_t i = 0; i < ny; ++i) {
      if (!std::isfinite(d->Y_host[i + a * d->ldy])) return bad("Y has a non-finite entry");
      if (d->Omega_host[i + a * d->ldo] > 1) return bad("Omega entries must be 0 or 1");
    }
  }

  cr_problem* p = new cr_problem();
  p->nx = (int)nx;
  p->ny = (int)ny;
  p->m = (int)m;
  p->rcap = opt.r_cap;
  p->lam = d->lambda;
  p->opt = opt;
  auto abort_create = [&](cr_status s) {
    g_create_err = p->err;
    cr_destroy(p);
    return s;
  };
  if (opt.stream) {
    p->st = (cudaStream_t)opt.stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess) {
      p->err = "cudaStreamCreate failed";
      return abort_create(CR_ECUDA);
    }
    p->own_stream = true;
  }
  p->launch_base = cr::g_launches.load();
  if (cudaMallocHost(&p->hs, sizeof(HostScal)) != cudaSuccess) {
    p->err = "cudaMallocHost failed";
    return abort_create(CR_ENOMEM);
  }
  cr_status s;
#define CK(x)                           \
  do {                                  \
    if ((s = (x)) != CR_OK) return abort_create(s); \
  } while (0)
  CK(build_lap(p, d->Ly, p->Ly));
  CK(build_lap(p, d->Lx, p->Lx));
  if (opt.precond == CR_PRECOND_MULTIGRID || opt.precond == CR_PRECOND_AUTO) {
    CK(build_mg(p, d->Ly, p->Ly, p->mg[0]));
    CK(build_mg(p, d->Lx, p->Lx, p->mg[1]));
  }
  // X: CSC, CSR by rows, and per-CTA local CSC on the x partition
  {
    std::vector<int> cp(m + 1, 0), row;
    std::vector<double> val;
    std::vector<std::vector<std::pair<int, double>>> byrow(nx);
    for (int64_t a = 0; a < m; ++a) {
      for (int64_t i = 0; i < nx; ++i) {
        const double x = d->X_host[i + a * d->ldx];
        if (x != 0.0) {
          row.push_back((int)i);
          val.push_back(x);
          byrow[i].push_back({(int)a, x});
        }
      }
      cp[a + 1] = (int)row.size();
    }
    std::vector<int> rp(nx + 1, 0), rc;
    std::vector<double> rv;
    for (int64_t i = 0; i < nx; ++i) {
      for (auto& e : byrow[i]) {
        rc.push_back(e.first);
        rv.push_back(e.second);
      }
      rp[i + 1] = (int)rc.size();
    }
    const int C = p->Lx.csize, chunk = p->Lx.chunk;
    std::vector<int> lp((size_t)C * m + 1, 0), lr;
    std::vector<double> lv;
    for (int r = 0; r < C; ++r)
      for (int64_t a = 0; a < m; ++a) {
        for (int q = cp[a]; q < cp[a + 1]; ++q)
          if (row[q] / chunk == r) {
            lr.push_back(row[q] - r * chunk);
            lv.push_back(val[q]);
          }
        lp[(size_t)r * m + a + 1] = (int)lr.size();
      }
    CK(upload(p, &p->xc_ptr, cp));
    CK(upload(p, &p->xc_row, row));
    CK(upload(p, &p->xc_val, val));
    int *d_rp, *d_rc, *d_lp, *d_lr;
    double *d_rv, *d_lv;
    CK(upload(p, &d_rp, rp));
    CK(upload(p, &d_rc, rc));
    CK(upload(p, &d_rv, rv));
    CK(upload(p, &d_lp, lp));
    CK(upload(p, &d_lr, lr));
    CK(upload(p, &d_lv, lv));
    std::vector<float> lvf(lv.begin(), lv.end()), rvf(rv.begin(), rv.end());
    float *d_lvf, *d_rvf;
    CK(upload(p, &d_lvf, lvf));
    CK(upload(p, &d_rvf, rvf));
    p->xl = DevXLocal{d_lp, d_lr, d_lv, d_rp, d_rc, d_rv, d_lvf, d_rvf};
    if (p->mg[1].nlev > 0) {
      // |X_a|^2: the v side's mean data weight enters the multigrid shift
      std::vector<double> xn2(m, 0.0);
      for (int64_t a = 0; a < m; ++a)
        for (int q = cp[a]; q < cp[a + 1]; ++q) xn2[a] += val[q] * val[q];
      double* dx = nullptr;
      CK(upload(p, &dx, xn2));
      p->mg[1].xn2 = dx;
    }
  }
  // Omega o Y, Omega; norms |D|_F (via the m x m Gram products, all terms of
  // one sign pattern: |D|^2 = tr((OmY^T OmY)(X^T X))) and |Omega o Y|^2
  std::vector<double> omy((size_t)ny * m);
  std::vector<uint8_t> om((size_t)ny * m);
  for (int64_t a = 0; a < m; ++a)
    for (int64_t i = 0; i < ny; ++i) {
      om[i + a * ny] = d->Omega_host[i + a * d->ldo];
      omy[i + a * ny] = om[i + a * ny] ? d->Y_host[i + a * d->ldy] : 0.0;
    }
  {
    std::vector<double> g1((size_t)m * m, 0.0), g2((size_t)m * m, 0.0);
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = 0; b <= a; ++b) {
        double s1 = 0.0, s2 = 0.0;
        for (int64_t i = 0; i < ny; ++i) s1 += omy[i + a * ny] * omy[i + b * ny];
        for (int64_t i = 0; i < nx; ++i) s2 += d->X_host[i + a * d->ldx] * d->X_host[i + b * d->ldx];
        g1[a + b * m] = g1[b + a * m] = s1;
        g2[a + b * m] = g2[b + a * m] = s2;
      }
    double dn2 = 0.0, on2 = 0.0;
    for (size_t t = 0; t < g1.size(); ++t) dn2 += g1[t] * g2[t];
    for (int64_t a = 0; a < m; ++a) on2 += g1[a + a * m];
    p->Dnorm = std::sqrt(std::max(dn2, 0.0));
    p->OmYn2 = on2;
  }
  CK(upload(p, &p->OmY, omy));
  CK(upload(p, &p->Om, om));
  const int rc = p->rcap;
  const size_t r2 = (size_t)rc * rc;
  CK(dalloc(p, &p->UU, (size_t)3 * rc * ny));
  CK(dalloc(p, &p->VV, (size_t)3 * rc * nx));
  for (double** b : {&p->Z, &p->Zprev, &p->A1, &p->A2, &p->B1, &p->B2, &p->F, &p->gR, &p->gP, &p->gQ, &p->gZB2,
                     &p->gZB1, &p->gDg, &p->gT, &p->gzb})
    CK(dalloc(p, b, r2));
  for (double** b : {&p->H, &p->P, &p->Mzh, &p->gZH, &p->gGw}) CK(dalloc(p, b, (size_t)rc * m));
  CK(dalloc(p, &p->G, r2 * m));
  CK(dalloc(p, &p->E, (size_t)ny * m));
  CK(dalloc(p, &p->Bnm, (size_t)ny * std::max<int64_t>(m, 1) + (size_t)ny * m));
  const int nmax = (int)std::max(nx, ny);
  for (double** b : {&p->u, &p->uhat, &p->rhs_u, &p->tmpy}) CK(dalloc(p, b, ny));
  for (double** b : {&p->v, &p->vhat, &p->rhs_v, &p->tmpx}) CK(dalloc(p, b, nx));
  for (double** b : {&p->pr, &p->pp, &p->ps, &p->pw, &p->pdinv, &p->pomt, &p->fc_rold, &p->fc_d, &p->fc_t})
    CK(dalloc(p, b, nmax));
  CK(dalloc(p, &p->fc_y, m));
  for (double** b : {&p->xi, &p->eta, &p->svec}) CK(dalloc(p, b, m));
  CK(dalloc(p, &p->hc, (size_t)3 * rc + m));
  CK(dalloc(p, &p->gc, (size_t)3 * rc + m));
  CK(dalloc(p, &p->cvec, (size_t)3 * rc + 2 * m));
  CK(dalloc(p, &p->coef, 8));
  p->gal_nb = galerkin_grid_size();
  if (p->opt.galerkin_ctas > 0) p->gal_nb = std::min(p->gal_nb, (int)p->opt.galerkin_ctas);
  CK(dalloc(p, &p->gpart, (size_t)4 * std::max(1, p->gal_nb)));
  CK(dalloc(p, &p->gout, 4));
  CK(dalloc(p, &p->gbar, 2));
  CK(dalloc(p, &p->gerr, 1));
  if (p->gal_nb > 0 && opt.galerkin_form != CR_GALERKIN_JACOBI) {
    for (double** b : {&p->eQa, &p->eQa2, &p->eQb, &p->eQb2, &p->eA2t, &p->eB2t, &p->eFt, &p->eZt, &p->eDen,
                       &p->eTmp})
      CK(dalloc(p, b, r2));
    for (double** b : {&p->eHt, &p->eY, &p->eGt}) CK(dalloc(p, b, (size_t)rc * m));
    for (double** b : {&p->ela, &p->elb}) CK(dalloc(p, b, rc));
    CK(dalloc(p, &p->eg, m));
    for (double** b : {&p->eDl, &p->eZz, &p->eYd}) CK(dalloc(p, b, r2));
    for (double** b : {&p->eHg, &p->eS}) CK(dalloc(p, b, (size_t)rc * m));
    if (m <= 128) CK(dalloc(p, &p->eCi, (size_t)rc * m * m));
    CK(dalloc(p, &p->eW, 2 * r2));
    CK(dalloc(p, &p->ebord, 2 * ((size_t)rc + 1)));
    CK(dalloc(p, &p->earw, 2 * arrow_work_doubles(rc)));
    if (opt.precision == CR_MIXED) {
      for (float** b : {&p->fQa, &p->fZz}) CK(dalloc(p, b, r2));
      for (float** b : {&p->fla, &p->flb}) CK(dalloc(p, b, rc));
      for (float** b : {&p->fY, &p->fGt}) CK(dalloc(p, b, (size_t)rc * m));
    }
  }
  if (opt.precision == CR_MIXED) {
    for (float** b : {&p->fA1, &p->fA2, &p->fB1, &p->fB2, &p->fDg, &p->fF, &p->fZ, &p->fR, &p->fPa, &p->fPb, &p->fQ,
                      &p->fT2, &p->fT1, &p->fzb})
      CK(dalloc(p, b, r2));
    for (float** b : {&p->fH, &p->fTH, &p->fGw}) CK(dalloc(p, b, (size_t)rc * m));
    CK(dalloc(p, &p->fG, r2 * m));
    if (rc <= 128) {
      p->ldb = ((int64_t)ny + 63) / 64 * 64;
      uint16_t *h16 = nullptr, *l16 = nullptr;
      CK(dalloc(p, &h16, (size_t)p->ldb * 128));
      CK(dalloc(p, &l16, (size_t)p->ldb * 128));
      p->ubhi = h16;
      p->ublo = l16;
      p->tc_splits = std::max(1, std::min((int)((ny + 63) / 64), (2 * 152 + (int)m - 1) / (int)m));
      CK(dalloc(p, &p->tcpart, tc_part_elems(p->tc_splits, (int)m)));
      CK(dalloc(p, &p->tcerr, 1));
    }
  }
  CK(dalloc(p, &p->stat, 2));
  CK(dalloc(p, &p->ds, DS_COUNT));
  // residual-norm bases and core workspaces
  p->ldcl = 3 * (int64_t)rc;
  p->ldcr = m + 3 * (int64_t)rc;
  p->ldcx = 3 * (int64_t)rc;
  p->ldcp = 3 * (int64_t)rc + m;
  p->ldm = m + 3 * (int64_t)rc;
  CK(dalloc(p, &p->QL, (size_t)ny * (3 * rc + m)));
  CK(dalloc(p, &p->CL, (size_t)p->ldcl * 3 * rc));
  CK(dalloc(p, &p->QR, (size_t)nx * (3 * rc + m)));
  CK(dalloc(p, &p->CRm, (size_t)p->ldcr * p->ldcr));
  CK(dalloc(p, &p->Cx, (size_t)p->ldcx * m));
  CK(dalloc(p, &p->Cx2, (size_t)p->ldcx * m));
  CK(dalloc(p, &p->Ep, (size_t)ny * m));
  CK(dalloc(p, &p->CE, (size_t)m * m));
  CK(dalloc(p, &p->CP, (size_t)p->ldcp * p->ldm));
  CK(dalloc(p, &p->T1, (size_t)p->ldcp * p->ldm));
  CK(dalloc(p, &p->T2, (size_t)p->ldcp * p->ldm));
  CK(dalloc(p, &p->gram, (size_t)m * m));
  CK(dalloc(p, &p->tmat, (size_t)m * m));
  p->ws_elems = std::max<size_t>((size_t)8 * p->ldcp * p->ldm, (size_t)16 * (3 * rc + m) * m);
  p->ws_elems = std::max<size_t>(p->ws_elems, (size_t)16 * r2);
  CK(dalloc(p, &p->ws, p->ws_elems));
  // right residual basis: X first (host Gram-Schmidt twice, columns in X's span rejected)
  {
    std::vector<double> Q((size_t)nx * m, 0.0), Cm((size_t)p->ldcr * m, 0.0);
    int nq = 0;
    std::vector<double> w(nx);
    for (int64_t a = 0; a < m; ++a) {
      for (int64_t i = 0; i < nx; ++i) w[i] = d->X_host[i + a * d->ldx];
      double nb = 0.0;
      for (double x : w) nb += x * x;
      for (int pass = 0; pass < 2; ++pass)
        for (int q = 0; q < nq; ++q) {
          double c = 0.0;
          for (int64_t i = 0; i < nx; ++i) c += Q[i + (size_t)q * nx] * w[i];
          for (int64_t i = 0; i < nx; ++i) w[i] -= c * Q[i + (size_t)q * nx];
        }
      double na = 0.0;
      for (double x : w) na += x * x;
      if (nb > 0.0 && std::sqrt(na / nb) > 1e-12) {
        const double inv = 1.0 / std::sqrt(na);
        for (int64_t i = 0; i < nx; ++i) Q[i + (size_t)nq * nx] = w[i] * inv;
        ++nq;
      }
    }
    for (int64_t a = 0; a < m; ++a)
      for (int q = 0; q < nq; ++q) {
        double c = 0.0;
        for (int64_t i = 0; i < nx; ++i) c += Q[i + (size_t)q * nx] * d->X_host[i + a * d->ldx];
        Cm[q + (size_t)a * p->ldcr] = c;
      }
    CUCHK(p, cudaMemcpyAsync(p->QR, Q.data(), sizeof(double) * nx * nq, cudaMemcpyHostToDevice, p->st));
    p->h2d_bytes += (int64_t)(sizeof(double) * nx * nq);
    CUCHK(p, cudaMemcpyAsync(p->CRm, Cm.data(), sizeof(double) * Cm.size(), cudaMemcpyHostToDevice, p->st));
    p->h2d_bytes += (int64_t)(sizeof(double) * Cm.size());
    p->nQR = nq;
    p->nQX = nq;
    if (sync(p) != CR_OK) return abort_create(CR_ECUDA);
  }
  refresh_E(p);
  if ((s = sync(p)) != CR_OK) return abort_create(s);
  if (d->grid_y.box_index) CK(cr_set_voxel_grid(p, 0, d->grid_y.dims, d->grid_y.box_index));
  if (d->grid_x.box_index) CK(cr_set_voxel_grid(p, 1, d->grid_x.dims, d->grid_x.box_index));
#undef CK
  *out = p;
  return CR_OK;
}

cr_status cr_add_rank_one(cr_problem* p, cr_rank1_info* info) {
  if (!p) return CR_EINVAL;
  return do_rank_one(p, info);
}

cr_status cr_project(cr_problem* p, double tol, cr_proj_info* info) {
  if (!p || !(tol >= 0.0)) return CR_EINVAL;
  return do_project(p, tol, info);
}

cr_status cr_residual(cr_problem* p, double* relres, double* J, double* dW) {
  if (!p) return CR_EINVAL;
  prof_begin(p, CR_PHASE_RESID);
  const int j = p->j;
  const int64_t ld = p->rcap;
  if (dW) {
    if (j == 0) {
      *dW = 0.0;
    } else {
      mat_diff_norms(j, p->Z, p->Zprev, ld, p->ds + DS_DW, p->st);
      TRY(readback(p, DS_DW, 2, false));
      const double a = p->hs->ds[DS_DW], b = p->hs->ds[DS_DW + 1];
      *dW = b > 0.0 ? std::sqrt(a / b) : 0.0;
    }
  }
  if (J) {
    if (j == 0) {
      *J = 0.5 * p->OmYn2;
    } else {
      if (!p->F_valid) build_F(p);
      galerkin_apply(p, p->Z, p->gQ);
      mat_dot(j, j, p->Z, ld, p->gQ, ld, p->ds + DS_ZKZ, p->st);
      mat_dot(j, j, p->Z, ld, p->F, ld, p->ds + DS_ZF, p->st);
      TRY(readback(p, DS_ZKZ, 2, false));
      *J = 0.5 * p->hs->ds[DS_ZKZ] - p->hs->ds[DS_ZF] + 0.5 * p->OmYn2;
    }
  }
  if (relres) TRY(do_relres(p, relres));
  prof_end(p, CR_PHASE_RESID);
  return CR_OK;
}

cr_status cr_set_voxel_grid(cr_problem* p, int32_t side, const int32_t* dims, const int32_t* box_index) {
  if (!p || (side != 0 && side != 1) || !dims || !box_index) return CR_EINVAL;
  const int n = side == 0 ? p->ny : p->nx;
  std::string err;
  if (!grid_ok(dims, box_index, n, err)) return fail(p, CR_EINVAL, err);
  std::vector<int> idx(box_index, box_index + n);
  int* d = nullptr;
  TRY(upload(p, &d, idx));
  p->box[side] = d;
  for (int k = 0; k < 3; ++k) p->box_dims[side][k] = dims[k];
  return sync(p);
}

cr_status cr_set_preconditioner(cr_problem* p, cr_net* net) {
  if (!p) return CR_EINVAL;
  if (!net) {
    p->net = nullptr;
    return CR_OK;
  }
  const int64_t V = net_voxels(net);
  for (int s = 0; s < 2; ++s)
    if (p->box[s] && (int64_t)p->box_dims[s][0] * p->box_dims[s][1] * p->box_dims[s][2] != V)
      return fail(p, CR_EINVAL, "network box does not match the voxel grid");
  if (p->net_V != V) {
    TRY(dalloc(p, &p->net_in, (size_t)2 * V));
    TRY(dalloc(p, &p->net_out, (size_t)V));
    p->net_V = V;
  }
  p->net = net;
  for (int s = 0; s < 2; ++s) {
    p->jac_iters[s] = p->learned_streak[s] = 0;
    p->jac_sec[s] = 0.0;
    p->learned_off[s] = false;
  }
  return sync(p);
}

cr_status cr_galerkin_assembly(cr_problem* p, int32_t method, float* G_host, int64_t ldg) {
  if (!p || !G_host) return CR_EINVAL;
  const int j = p->j;
  if (j == 0) return CR_OK;
  if (ldg < j) return fail(p, CR_EINVAL, "ldg < rank");
  if (!p->fG) return fail(p, CR_ESTATE, "the assembly runs in the mixed form (precision = CR_MIXED)");
  if (method == 0 && !(p->ubhi && j <= 128)) return fail(p, CR_EINVAL, "tensor-core assembly needs r_cap <= 128");
  if (p->tcerr) CUCHK(p, cudaMemsetAsync(p->tcerr, 0, sizeof(int), p->st));
  TRY(mixed_G(p, method == 0));
  int herr = 0;
  if (p->tcerr) CUCHK(p, cudaMemcpyAsync(&herr, p->tcerr, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  const int64_t ld = p->rcap;
  for (int a = 0; a < p->m; ++a)
    CUCHK(p, cudaMemcpy2DAsync(G_host + (size_t)a * ldg * j, ldg * sizeof(float), p->fG + (size_t)a * ld * ld,
                               ld * sizeof(float), j * sizeof(float), j, cudaMemcpyDeviceToHost, p->st));
  p->d2h_bytes += (int64_t)sizeof(float) * p->m * j * j;
  TRY(sync(p));
  if (herr)
    return fail(p, CR_ETIMEOUT, "tensor-core assembly: an mbarrier wait timed out (site*100000 + K-block + 1 = " +
                                    std::to_string(herr) + ")");
  return CR_OK;
}

cr_status cr_get_stats(cr_problem* p, cr_stats* s, int32_t reset) {
  if (!p || !s) return CR_EINVAL;
  CUCHK(p, cudaStreamSynchronize(p->st));
  prof_resolve(p);
  std::memset(s, 0, sizeof(*s));
  s->launches = cr::g_launches.load() - p->launch_base;
  s->pcg_solves = p->pcg_solves;
  s->pcg_iters = p->pcg_iters;
  s->h2d_bytes = p->h2d_bytes;
  s->d2h_bytes = p->d2h_bytes;
  s->learned_solves = p->learned_solves;
  s->learned_fallbacks = p->fcg_fallbacks;
  s->learned_off = (p->learned_off[0] ? 1 : 0) | (p->learned_off[1] ? 2 : 0);
  s->mixed_handovers = p->mixed_handovers;
  for (int side = 0; side < 2; ++side) {
    const DevLap& L = side == 0 ? p->Ly : p->Lx;
    const bool f32 = p->opt.precision == CR_MIXED;
    s->pcg_cluster[side] = (use_mg(p, side, f32) || !use_grid_pcg(p, side, f32)) ? L.csize : 0;
    s->pcg_multigrid[side] = use_mg(p, side, f32) ? p->mg[side].nlev : 0;
  }
  s->galerkin_eigen[0] = p->gal_eig_proj;
  s->galerkin_eigen[1] = p->gal_eig_finish;
  for (int side = 0; side < 2; ++side) {
    const bool f32 = p->opt.precision == CR_MIXED;
    const double w = f32 ? 4.0 : 8.0;
    const DevLap& L = side == 0 ? p->Ly : p->Lx;
    s->pcg_iters_side[side] = p->pcg_iters_side[side];
    double b = (double)L.n * (10.0 * w + 4.0 * L.K);  // Jacobi PCG (Chronopoulos-Gear)
    if (use_mg(p, side, f32)) {
      b = p->mg[side].bytes_iter[f32 ? 0 : 1];
      if (side == 1 && p->mg[1].smw) b += (double)L.n * p->m * w;  // the Woodbury correction reads M0^-1 X
    }
    s->pcg_bytes_per_iter[side] = b;
  }
  for (int i = 0; i < CR_NPHASE; ++i) {
    s->phase_ms[i] = p->phase_ms[i];
    s->phase_calls[i] = p->phase_calls[i];
  }
  if (reset) {
    p->launch_base = cr::g_launches.load();
    p->pcg_solves = p->pcg_iters = 0;
    p->pcg_iters_side[0] = p->pcg_iters_side[1] = 0;
    p->h2d_bytes = p->d2h_bytes = 0;
    p->learned_solves = p->fcg_fallbacks = p->mixed_handovers = 0;
    p->gal_eig_proj = p->gal_eig_finish = 0;
    for (int i = 0; i < CR_NPHASE; ++i) {
      p->phase_ms[i] = 0.0;
      p->phase_calls[i] = 0;
    }
  }
  return CR_OK;
}

cr_status cr_solve(cr_problem* p, int32_t r_max, double tau, double relres_target, cr_solve_info* info) {
  if (!p || r_max < 0 || !(tau >= 0.0)) return CR_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  cr_solve_info si{};
  si.stop = CR_STOP_NONE;
  si.relres = NAN;
  si.dW = NAN;
  cr_status rc = CR_OK;
  int step = 0;
  // residual_every == 0: the checks follow relres's observed decay.  After a check
  // the rate per step from the previous one predicts the steps left to the target;
  // the next check comes after half of them (1 to kMaxGap steps), so checks are
  // sparse far from the target and every step close to it.
  constexpr int kMaxGap = 32;
  int next_check = 1, last_step = 0;
  double last_rr = 0.0;
  while (p->j < std::min(r_max, p->rcap)) {
    cr_rank1_info ri{};
    cr_status s = do_rank_one(p, &ri);
    si.pcg_iters += ri.pcg_iters_u + ri.pcg_iters_v;
    if (s == CR_ERANK) {
      si.stop = CR_STOP_RANK;
      break;
    }
    if (s != CR_OK && s != CR_ENOTCONV) return s;
    if (s == CR_ENOTCONV) rc = s;
    cr_proj_info pi{};
    s = do_project(p, tau / 2.0, &pi);
    si.cg_iters += pi.iters;
    if (s != CR_OK && s != CR_ENOTCONV) return s;
    if (s == CR_ENOTCONV) rc = s;
    ++step;
    double dW = 0.0;
    double* rr = nullptr;
    double relres = NAN;
    const bool due = p->opt.residual_every == 0 ? step >= next_check
                                                : step % std::max(1, p->opt.residual_every) == 0;
    if (relres_target > 0.0 && (due || p->j >= r_max)) rr = &relres;
    TRY(cr_residual(p, rr, nullptr, &dW));
    si.dW = dW;
    if (rr) {
      si.relres = relres;
      int gap = 1;
      if (last_rr > 0.0 && relres > relres_target && relres < last_rr && step > last_step) {
        const double rate = std::log(last_rr / relres) / (step - last_step);
        const double left = std::log(relres / relres_target) / rate;
        gap = (int)std::max(1.0, std::min((double)kMaxGap, std::floor(0.5 * left)));
      }
      next_check = step + gap;
      last_rr = relres;
      last_step = step;
    }
    if (dW <= tau) {
      si.stop = CR_STOP_DW;
      break;
    }
    if (rr && relres <= relres_target) {
      si.stop = CR_STOP_RELRES;
      break;
    }
  }
  if (si.stop == CR_STOP_NONE) si.stop = CR_STOP_RMAX;
  si.rank = p->j;
  double J = NAN;
  TRY(cr_residual(p, std::isnan(si.relres) ? &si.relres : nullptr, &J, nullptr));
  si.J = J;
  si.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = si;
  return rc;
}

cr_status cr_get_rank(const cr_problem* p, int32_t* j) {
  if (!p || !j) return CR_EINVAL;
  *j = p->j;
  return CR_OK;
}

cr_status cr_get_factors(cr_problem* p, double* U, int64_t ldu, double* Zh, int64_t ldz, double* V, int64_t ldv) {
  if (!p) return CR_EINVAL;
  const int j = p->j;
  if (j == 0) return CR_OK;
  if ((U && ldu < p->ny) || (Zh && ldz < j) || (V && ldv < p->nx)) return fail(p, CR_EINVAL, "leading dimension");
  p->d2h_bytes += (int64_t)sizeof(double) * ((U ? (int64_t)p->ny * j : 0) + (V ? (int64_t)p->nx * j : 0) +
                                             (Zh ? (int64_t)j * j : 0));
  if (U)
    CUCHK(p, cudaMemcpy2DAsync(U, ldu * sizeof(double), p->UU, 3 * (size_t)p->ny * sizeof(double),
                               p->ny * sizeof(double), j, cudaMemcpyDeviceToHost, p->st));
  if (V)
    CUCHK(p, cudaMemcpy2DAsync(V, ldv * sizeof(double), p->VV, 3 * (size_t)p->nx * sizeof(double),
                               p->nx * sizeof(double), j, cudaMemcpyDeviceToHost, p->st));
  if (Zh)
    CUCHK(p, cudaMemcpy2DAsync(Zh, ldz * sizeof(double), p->Z, (size_t)p->rcap * sizeof(double), j * sizeof(double),
                               j, cudaMemcpyDeviceToHost, p->st));
  return sync(p);
}

namespace {
// Checkpoint layout: StateHeader, then U (ny x j), Z (j x j), Z of the step before (j x j), V (nx x j),
// float64 column-major, contiguous.
struct StateHeader {
  char magic[8];
  int64_t ny, nx, m, j;
  double lam;
  uint64_t checksum;  // FNV-1a of the payload bytes
};
constexpr char kStateMagic[8] = {'C', 'R', 'S', 'T', 'A', 'T', 'E', '1'};

uint64_t fnv1a(const unsigned char* b, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

size_t state_bytes(int64_t ny, int64_t nx, int64_t j) {
  return sizeof(StateHeader) + sizeof(double) * (size_t)(ny * j + 2 * j * j + nx * j);
}
}  // namespace

cr_status cr_get_state(cr_problem* p, void* buf, size_t* bytes) {
  if (!p || !bytes) return CR_EINVAL;
  const int j = p->j;
  const size_t need = state_bytes(p->ny, p->nx, j);
  if (!buf) {
    *bytes = need;
    return CR_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return fail(p, CR_EINVAL, "state buffer too small (" + std::to_string(need) + " bytes needed)");
  }
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.ny = p->ny;
  h.nx = p->nx;
  h.m = p->m;
  h.j = j;
  h.lam = p->lam;
  unsigned char* out = static_cast<unsigned char*>(buf);
  double* U = reinterpret_cast<double*>(out + sizeof(StateHeader));
  double* Z = U + (size_t)p->ny * j;
  double* Zp = Z + (size_t)j * j;
  double* V = Zp + (size_t)j * j;
  if (j > 0) {
    TRY(cr_get_factors(p, U, p->ny, Z, j, V, p->nx));
    CUCHK(p, cudaMemcpy2DAsync(Zp, j * sizeof(double), p->Zprev, (size_t)p->rcap * sizeof(double), j * sizeof(double),
                               j, cudaMemcpyDeviceToHost, p->st));
    p->d2h_bytes += (int64_t)sizeof(double) * j * j;
    TRY(sync(p));
  }
  h.checksum = fnv1a(out + sizeof(StateHeader), need - sizeof(StateHeader));
  std::memcpy(out, &h, sizeof(h));
  *bytes = need;
  return CR_OK;
}

cr_status cr_set_state(cr_problem* p, const void* buf, size_t bytes) {
  if (!p || !buf) return CR_EINVAL;
  if (bytes < sizeof(StateHeader)) return fail(p, CR_EINVAL, "state buffer shorter than its header");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, 8) != 0) return fail(p, CR_EINVAL, "not a cr_get_state buffer");
  if (h.ny != p->ny || h.nx != p->nx || h.m != p->m || std::memcmp(&h.lam, &p->lam, sizeof(double)) != 0)
    return fail(p, CR_EINVAL, "state belongs to a problem with other sizes or another lambda");
  if (h.j < 0 || h.j > (int64_t)std::min(p->ny, p->nx)) return fail(p, CR_EINVAL, "corrupt state (rank)");
  if (h.j > p->rcap) return fail(p, CR_ESTATE, "state rank exceeds r_cap");
  const int j = (int)h.j;
  const size_t need = state_bytes(p->ny, p->nx, j);
  if (bytes < need) return fail(p, CR_EINVAL, "state buffer truncated");
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  if (fnv1a(in + sizeof(StateHeader), need - sizeof(StateHeader)) != h.checksum)
    return fail(p, CR_EINVAL, "state checksum mismatch (corrupt buffer)");
  // the payload may sit at any alignment in the caller's buffer
  std::vector<double> pay((need - sizeof(StateHeader)) / sizeof(double));
  std::memcpy(pay.data(), in + sizeof(StateHeader), need - sizeof(StateHeader));
  const double* U = pay.data();
  const double* Z = U + (size_t)p->ny * j;
  const double* Zp = Z + (size_t)j * j;
  const double* V = Zp + (size_t)j * j;
  TRY(cr_set_factors(p, j, j ? U : nullptr, p->ny, j ? Z : nullptr, std::max(j, 1), j ? V : nullptr, p->nx));
  if (j > 0) {
    CUCHK(p, cudaMemcpy2DAsync(p->Zprev, (size_t)p->rcap * sizeof(double), Zp, j * sizeof(double), j * sizeof(double),
                               j, cudaMemcpyHostToDevice, p->st));
    p->h2d_bytes += (int64_t)sizeof(double) * j * j;
  }
  return sync(p);
}

cr_status cr_set_factors(cr_problem* p, int32_t j, const double* U, int64_t ldu, const double* Zh, int64_t ldz,
                         const double* V, int64_t ldv) {
  if (!p) return CR_EINVAL;
  if (j < 0 || j > p->rcap) return fail(p, CR_EINVAL, "rank outside [0, r_cap]");
  if (j > 0 && (!U || !Zh || !V || ldu < p->ny || ldz < j || ldv < p->nx))
    return fail(p, CR_EINVAL, "null factor or leading dimension too small");
  cudaStream_t st = p->st;
  const int64_t ld = p->rcap;
  fill((int64_t)ld * ld, 0.0, p->Z, st);
  fill((int64_t)p->ldcl * 3 * ld, 0.0, p->CL, st);
  fill((int64_t)p->ldcr * p->ldcr - (int64_t)p->ldcr * p->m, 0.0, p->CRm + (size_t)p->ldcr * p->m, st);
  p->nQL = 0;
  p->nQR = p->nQX;  // the X part of the right basis does not depend on the factors
  p->qr_step.clear();
  p->j = 0;
  eig_reset(p);
  if (j > 0) {
    CUCHK(p, cudaMemcpy2DAsync(p->UU, 3 * (size_t)p->ny * sizeof(double), U, ldu * sizeof(double),
                               p->ny * sizeof(double), j, cudaMemcpyHostToDevice, st));
    CUCHK(p, cudaMemcpy2DAsync(p->VV, 3 * (size_t)p->nx * sizeof(double), V, ldv * sizeof(double),
                               p->nx * sizeof(double), j, cudaMemcpyHostToDevice, st));
    CUCHK(p, cudaMemcpy2DAsync(p->Z, ld * sizeof(double), Zh, ldz * sizeof(double), j * sizeof(double), j,
                               cudaMemcpyHostToDevice, st));
    for (int q = 0; q < j; ++q) TRY(grow_projections(p, q));
  }
  p->j = j;
  CUCHK(p, cudaMemcpyAsync(p->Zprev, p->Z, sizeof(double) * ld * ld, cudaMemcpyDeviceToDevice, st));
  build_F(p);
  refresh_E(p);
  return sync(p);
}

cr_status cr_cv_error(cr_problem* p, int32_t mt, const double* Xt, int64_t ldx, const double* Yt, int64_t ldy,
                      const uint8_t* Omt, int64_t ldo, double* num, double* den) {
  if (!p || !num || !den || mt < 0) return CR_EINVAL;
  *num = *den = 0.0;
  if (mt == 0) return CR_OK;
  if (!Xt || !Yt || !Omt || ldx < p->nx || ldy < p->ny || ldo < p->ny) return fail(p, CR_EINVAL, "held-out data");
  const int nx = p->nx, ny = p->ny, j = p->j;
  cudaStream_t st = p->st;
  if (mt > p->cv_cap) {
    const int c = std::max(mt, 2 * p->cv_cap);
    TRY(dalloc(p, &p->cv_X, (size_t)nx * c));
    TRY(dalloc(p, &p->cv_Y, (size_t)ny * c));
    TRY(dalloc(p, &p->cv_P, (size_t)ny * c));
    TRY(dalloc(p, &p->cv_T1, (size_t)p->rcap * c));
    TRY(dalloc(p, &p->cv_T2, (size_t)p->rcap * c));
    TRY(dalloc(p, &p->cv_Om, (size_t)ny * c));
    if (!p->cv_out) TRY(dalloc(p, &p->cv_out, 2));
    p->cv_cap = c;
  }
  CUCHK(p, cudaMemcpy2DAsync(p->cv_X, nx * sizeof(double), Xt, ldx * sizeof(double), nx * sizeof(double), mt,
                             cudaMemcpyHostToDevice, st));
  CUCHK(p, cudaMemcpy2DAsync(p->cv_Y, ny * sizeof(double), Yt, ldy * sizeof(double), ny * sizeof(double), mt,
                             cudaMemcpyHostToDevice, st));
  CUCHK(p, cudaMemcpy2DAsync(p->cv_Om, ny, Omt, ldo, ny, mt, cudaMemcpyHostToDevice, st));
  p->h2d_bytes += (int64_t)mt * (nx * 8 + ny * 9);
  if (j == 0) {
    fill((int64_t)ny * mt, 0.0, p->cv_P, st);
  } else {
    // T1 = V^T X_t (j x mt), T2 = Z T1, P = U T2 (U, V: column p at 3p of the interleaved panels)
    gemm(j, mt, nx, 1.0, MatView{p->VV, 3 * (int64_t)nx, 1}, MatView{p->cv_X, 1, nx}, 0.0, p->cv_T1, 1, j, p->ws,
         p->ws_elems, st);
    gemm(j, mt, j, 1.0, MatView{p->Z, 1, p->rcap}, MatView{p->cv_T1, 1, j}, 0.0, p->cv_T2, 1, j, p->ws, p->ws_elems,
         st);
    gemm(ny, mt, j, 1.0, MatView{p->UU, 1, 3 * (int64_t)ny}, MatView{p->cv_T2, 1, j}, 0.0, p->cv_P, 1, ny, p->ws,
         p->ws_elems, st);
  }
  cv_err(ny, mt, p->cv_P, p->cv_Y, p->cv_Om, p->cv_out, st);
  double out[2] = {0.0, 0.0};
  CUCHK(p, cudaMemcpyAsync(out, p->cv_out, sizeof(out), cudaMemcpyDeviceToHost, st));
  p->d2h_bytes += (int64_t)sizeof(out);
  TRY(sync(p));
  *num = out[0];
  *den = out[1];
  return CR_OK;
}

cr_status cr_svd_factors(cr_problem* p, double* Uh, int64_t ldu, double* sigma, double* Vh, int64_t ldv) {
  if (!p) return CR_EINVAL;
  const int j = p->j, ny = p->ny, nx = p->nx;
  if (j == 0) return CR_OK;
  if ((Uh && ldu < ny) || (Vh && ldv < nx)) return fail(p, CR_EINVAL, "leading dimension");
  cudaStream_t st = p->st;
  // the core Z to the host, its SVD there (j x j), then U^ = U U~ and V^ = V V~ on the device
  std::vector<double> A((size_t)j * j), s, Vt;
  CUCHK(p, cudaMemcpy2DAsync(A.data(), j * sizeof(double), p->Z, (size_t)p->rcap * sizeof(double),
                             j * sizeof(double), j, cudaMemcpyDeviceToHost, st));
  p->d2h_bytes += (int64_t)sizeof(double) * j * j;
  TRY(sync(p));
  jacobi_svd(j, A, s, Vt);
  if (sigma) std::copy(s.begin(), s.end(), sigma);
  if (!Uh && !Vh) return CR_OK;
  if (!p->post_small) TRY(dalloc(p, &p->post_small, (size_t)2 * p->rcap * p->rcap));
  double* dUt = p->post_small;
  double* dVt = p->post_small + (size_t)p->rcap * p->rcap;
  if (Uh) {
    if (!p->post_Uh) TRY(dalloc(p, &p->post_Uh, (size_t)ny * p->rcap));
    CUCHK(p, cudaMemcpyAsync(dUt, A.data(), sizeof(double) * j * j, cudaMemcpyHostToDevice, st));
    gemm(ny, j, j, 1.0, MatView{p->UU, 1, 3 * (int64_t)ny}, MatView{dUt, 1, j}, 0.0, p->post_Uh, 1, ny, p->ws,
         p->ws_elems, st);
    CUCHK(p, cudaMemcpy2DAsync(Uh, ldu * sizeof(double), p->post_Uh, ny * sizeof(double), ny * sizeof(double), j,
                               cudaMemcpyDeviceToHost, st));
    p->h2d_bytes += (int64_t)sizeof(double) * j * j;
    p->d2h_bytes += (int64_t)sizeof(double) * ny * j;
  }
  if (Vh) {
    if (!p->post_Vh) TRY(dalloc(p, &p->post_Vh, (size_t)nx * p->rcap));
    CUCHK(p, cudaMemcpyAsync(dVt, Vt.data(), sizeof(double) * j * j, cudaMemcpyHostToDevice, st));
    gemm(nx, j, j, 1.0, MatView{p->VV, 1, 3 * (int64_t)nx}, MatView{dVt, 1, j}, 0.0, p->post_Vh, 1, nx, p->ws,
         p->ws_elems, st);
    CUCHK(p, cudaMemcpy2DAsync(Vh, ldv * sizeof(double), p->post_Vh, nx * sizeof(double), nx * sizeof(double), j,
                               cudaMemcpyDeviceToHost, st));
    p->h2d_bytes += (int64_t)sizeof(double) * j * j;
    p->d2h_bytes += (int64_t)sizeof(double) * nx * j;
  }
  return sync(p);
}

cr_status cr_solution_report(cr_problem* p, int32_t nonneg, int32_t jr, const double* Ur, int64_t ldur,
                             const double* Zr, int64_t ldzr, const double* Vr, int64_t ldvr, double* W, int64_t ldw,
                             cr_solution_stats* out) {
  if (!p || !out) return CR_EINVAL;
  *out = cr_solution_stats{};
  const int ny = p->ny, nx = p->nx, j = p->j;
  if (jr < 0) return fail(p, CR_EINVAL, "reference rank below zero");
  if (jr > 0 && (!Ur || !Zr || !Vr || ldur < ny || ldzr < jr || ldvr < nx))
    return fail(p, CR_EINVAL, "reference factors: null pointer or leading dimension too small");
  if (W && ldw < ny) return fail(p, CR_EINVAL, "leading dimension of W");
  cudaStream_t st = p->st;
  out->entries = (int64_t)ny * nx;
  if (out->entries == 0) return CR_OK;
  // P = U Z (ny x j); U's columns sit every third column of the interleaved panel
  if (!p->post_P) TRY(dalloc(p, &p->post_P, (size_t)ny * p->rcap));
  if (j > 0)
    gemm(ny, j, j, 1.0, MatView{p->UU, 1, 3 * (int64_t)ny}, MatView{p->Z, 1, p->rcap}, 0.0, p->post_P, 1, ny, p->ws,
         p->ws_elems, st);
  if (jr > 0) {
    if (jr > p->post_ref_cap) {
      const int c = std::max(jr, p->rcap);
      TRY(dalloc(p, &p->post_Ur, (size_t)ny * c));
      TRY(dalloc(p, &p->post_Zr, (size_t)c * c));
      TRY(dalloc(p, &p->post_Vr, (size_t)nx * c));
      TRY(dalloc(p, &p->post_Pr, (size_t)ny * c));
      p->post_ref_cap = c;
    }
    CUCHK(p, cudaMemcpy2DAsync(p->post_Ur, ny * sizeof(double), Ur, ldur * sizeof(double), ny * sizeof(double), jr,
                               cudaMemcpyHostToDevice, st));
    CUCHK(p, cudaMemcpy2DAsync(p->post_Zr, jr * sizeof(double), Zr, ldzr * sizeof(double), jr * sizeof(double), jr,
                               cudaMemcpyHostToDevice, st));
    CUCHK(p, cudaMemcpy2DAsync(p->post_Vr, nx * sizeof(double), Vr, ldvr * sizeof(double), nx * sizeof(double), jr,
                               cudaMemcpyHostToDevice, st));
    p->h2d_bytes += (int64_t)sizeof(double) * jr * ((int64_t)ny + nx + jr);
    gemm(ny, jr, jr, 1.0, MatView{p->post_Ur, 1, ny}, MatView{p->post_Zr, 1, jr}, 0.0, p->post_Pr, 1, ny, p->ws,
         p->ws_elems, st);
  }
  // without W on the host one launch covers every column; with it, blocks of
  // columns go through a device buffer of at most kPostBlockBytes
  constexpr int64_t kPostBlockBytes = (int64_t)256 << 20;
  int64_t cw = nx;
  if (W) {
    cw = std::max<int64_t>(64, kPostBlockBytes / ((int64_t)sizeof(double) * ny) / 64 * 64);
    cw = std::min<int64_t>(cw, nx);
    if (cw > p->post_W_cols) {
      TRY(dalloc(p, &p->post_W, (size_t)ny * cw));
      p->post_W_cols = cw;
    }
  }
  int64_t nparts = 0;
  for (int64_t c0 = 0; c0 < nx; c0 += cw) nparts += post_tiles_parts(ny, (int)std::min<int64_t>(cw, nx - c0));
  if (nparts > p->post_part_cap) {
    TRY(dalloc(p, &p->post_part, (size_t)nparts * PS_N));
    p->post_part_cap = nparts;
  }
  if (!p->post_out) TRY(dalloc(p, &p->post_out, PS_N));
  int64_t off = 0;
  for (int64_t c0 = 0; c0 < nx; c0 += cw) {
    const int ncols = (int)std::min<int64_t>(cw, nx - c0);
    post_tiles(ny, j, p->post_P, ny, p->VV, 3 * (int64_t)nx, jr, p->post_Pr, ny, p->post_Vr, nx, nonneg ? 1 : 0,
               (int)c0, ncols, W ? p->post_W : nullptr, ny, p->post_part + off * PS_N, st);
    off += post_tiles_parts(ny, ncols);
    if (W) {
      CUCHK(p, cudaMemcpy2DAsync(W + c0 * ldw, ldw * sizeof(double), p->post_W, ny * sizeof(double),
                                 ny * sizeof(double), ncols, cudaMemcpyDeviceToHost, st));
      p->d2h_bytes += (int64_t)sizeof(double) * ny * ncols;
    }
  }
  post_reduce((int)off, p->post_part, p->post_out, st);
  double r[PS_N];
  CUCHK(p, cudaMemcpyAsync(r, p->post_out, sizeof(r), cudaMemcpyDeviceToHost, st));
  p->d2h_bytes += (int64_t)sizeof(r);
  TRY(sync(p));
  out->n_negative = (int64_t)r[PS_NNEG];
  out->w_min = r[PS_MIN];
  out->w_max = r[PS_MAX];
  out->w_fro2 = r[PS_W2];
  out->neg_fro2 = r[PS_NEG2];
  out->ref_fro2 = r[PS_REF2];
  out->diff_fro2 = r[PS_DIFF2];
  out->diff_maxabs = r[PS_MAXABS];
  out->rms = std::sqrt(r[PS_DIFF2] / (double)out->entries);
  out->rel = r[PS_REF2] > 0.0 ? std::sqrt(r[PS_DIFF2] / r[PS_REF2]) : std::nan("");
  return CR_OK;
}

cr_status cr_apply_residual(cr_problem* p, int32_t trans, const double* in, double* out) {
  if (!p || !in || !out) return CR_EINVAL;
  cudaStream_t st = p->st;
  if (!trans) {
    CUCHK(p, cudaMemcpyAsync(p->tmpx, in, sizeof(double) * p->nx, cudaMemcpyHostToDevice, st));
    residual_times(p, p->tmpx, p->rhs_u);
    CUCHK(p, cudaMemcpyAsync(out, p->rhs_u, sizeof(double) * p->ny, cudaMemcpyDeviceToHost, st));
  } else {
    CUCHK(p, cudaMemcpyAsync(p->tmpy, in, sizeof(double) * p->ny, cudaMemcpyHostToDevice, st));
    residual_t_times(p, p->tmpy, p->rhs_v);
    CUCHK(p, cudaMemcpyAsync(out, p->rhs_v, sizeof(double) * p->nx, cudaMemcpyDeviceToHost, st));
  }
  return sync(p);
}

cr_status cr_solve_u(cr_problem* p, const double* v, const double* rhs, double* uh, int32_t* iters) {
  if (!p || !v || !rhs || !uh) return CR_EINVAL;
  cudaStream_t st = p->st;
  CUCHK(p, cudaMemcpyAsync(p->v, v, sizeof(double) * p->nx, cudaMemcpyHostToDevice, st));
  CUCHK(p, cudaMemcpyAsync(p->rhs_u, rhs, sizeof(double) * p->ny, cudaMemcpyHostToDevice, st));
  prep_u(p, p->v);
  fill(p->ny, 0.0, p->uhat, st);
  TRY(launch_pcg(p, 0, p->rhs_u, p->uhat));
  CUCHK(p, cudaMemcpyAsync(uh, p->uhat, sizeof(double) * p->ny, cudaMemcpyDeviceToHost, st));
  TRY(readback(p, 0, 1, true));
  if (iters) *iters = p->hs->stat[0].iters;
  if (p->hs->stat[0].status == 2) return fail(p, CR_ENOTCONV, "PCG breakdown");
  if (p->hs->stat[0].status == 1) return fail(p, CR_ENOTCONV, "PCG reached pcg_maxit");
  return CR_OK;
}

cr_status cr_solve_v(cr_problem* p, const double* u, const double* rhs, double* vh, int32_t* iters) {
  if (!p || !u || !rhs || !vh) return CR_EINVAL;
  cudaStream_t st = p->st;
  CUCHK(p, cudaMemcpyAsync(p->u, u, sizeof(double) * p->ny, cudaMemcpyHostToDevice, st));
  CUCHK(p, cudaMemcpyAsync(p->rhs_v, rhs, sizeof(double) * p->nx, cudaMemcpyHostToDevice, st));
  prep_v(p, p->u);
  fill(p->nx, 0.0, p->vhat, st);
  TRY(launch_pcg(p, 1, p->rhs_v, p->vhat));
  CUCHK(p, cudaMemcpyAsync(vh, p->vhat, sizeof(double) * p->nx, cudaMemcpyDeviceToHost, st));
  TRY(readback(p, 0, 1, true));
  if (iters) *iters = p->hs->stat[1].iters;
  if (p->hs->stat[1].status == 2) return fail(p, CR_ENOTCONV, "PCG breakdown");
  if (p->hs->stat[1].status == 1) return fail(p, CR_ENOTCONV, "PCG reached pcg_maxit");
  return CR_OK;
}

}  // extern "C"
