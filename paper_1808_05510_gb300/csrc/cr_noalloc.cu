// Allocation-free solve of the u-side ALS system for callers that cannot call
// cudaMalloc.
//
// Who needs it: code that runs where allocating device memory is not allowed
// or not possible -- inside a region whose memory budget is fixed up front
// (a plug-in handed only pre-sized buffers by its host application), on a
// thread that must not take the allocator's locks, or in a process whose
// allocator is owned by another runtime.  Such callers hold their inputs and
// outputs in memory they already own; this entry point needs nothing else.
//
// How: the work vectors of the PCG (residual, search directions, operator
// products, Jacobi diagonal) and its status words live in one file-scope
// static __device__ array sized for at most kMaxN rows.  Every GPU that loads
// the library keeps that array (about 5 MiB) until the process exits.  Host
// code cannot use the array's name as a device address, so every call (with
// the device current) looks the address up with cudaGetSymbolAddress and sets
// the kernel's launch attributes; both are cheap host calls and always refer
// to the current context, so a cudaDeviceReset between calls leaves nothing
// stale.  The first call on a device also loads the library's device code
// there.  All calls share the
// one array and it keeps the last call's contents: the status words are
// cleared before each launch, and two calls whose kernels overlap on the GPU
// (different streams, or several host threads) race on the array and produce
// garbage.  Each call waits for its stream to finish before it returns (it
// reads the status words back).
//
// The operator is the one of the existing u-side solve:
//   lam [(L + c I)^2 + (d - c^2) I] + diag(omega),
// with L given in CSR form in device memory; the iteration is the same
// cluster-resident Chronopoulos-Gear PCG with a Jacobi preconditioner,
// started from zero.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "conreg.h"
#include "cr_common.cuh"

namespace cg = cooperative_groups;

namespace cr {
void set_global_error(const std::string& msg);  // cr_api.cu
}

namespace {

constexpr int64_t kMaxN = 131072;     // rows (16 CTAs x 8192)
constexpr int kVecs = 5;              // r, p, s, w, dinv
constexpr int64_t kStatOff = kVecs * kMaxN;
constexpr int kThreads = 512;

static __device__ __align__(256) double g_scratch[kVecs * kMaxN + 8];

struct NaArgs {
  int n;
  const int* rp;
  const int* col;
  const double* val;
  double lam, c, d;
  const double* omega;
  const double* b;
  double* x;
  double* scratch;  // device address of g_scratch
  double tol;
  int maxit;
  int chunk;
};

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NV>
__device__ __forceinline__ void na_block_sum(double (&v)[NV], double* scr, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = na_warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) scr[wid * NV + q] = v[q];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = lane < nw ? scr[lane * NV + q] : 0.0;
      t = na_warp_sum(t);
      if (lane == 0) out[q] = t;
    }
  }
}

template <int NV>
__device__ __forceinline__ void na_cluster_sum(cg::cluster_group& cl, double* red, double* scal, int csize) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      if (lane < csize) t = cl.map_shared_rank(red, lane)[q];
      t = na_warp_sum(t);
      if (lane == 0) scal[q] = t;
    }
  }
  __syncthreads();
}

// ((L + shift I) v)_i with v in distributed shared memory, L in CSR.
__device__ __forceinline__ double na_row(const NaArgs& A, int i, double shift, double* buf, cg::cluster_group& cl) {
  double acc = 0.0;
  for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
    const int jj = A.col[q];
    const int owner = jj / A.chunk;
    const double vj = cl.map_shared_rank(buf, (unsigned)owner)[jj - owner * A.chunk];
    acc += A.val[q] * vj;
  }
  const int me = i / A.chunk;
  return acc + shift * cl.map_shared_rank(buf, (unsigned)me)[i - me * A.chunk];
}

__global__ void __launch_bounds__(kThreads, 1) na_pcg_kernel(const NaArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int chunk = A.chunk;
  const int beg = rank * chunk;
  const int nloc = max(0, min(A.n - beg, chunk));
  extern __shared__ __align__(16) double sm[];
  double* ub0 = sm;
  double* ub1 = sm + chunk;
  double* tb = sm + 2 * chunk;
  double* red = tb + chunk;  // [8]
  double* scr = red + 8;     // [128]
  double* scal = scr + 128;  // [8]
  double* r = A.scratch;
  double* p = A.scratch + kMaxN;
  double* s = A.scratch + 2 * kMaxN;
  double* w = A.scratch + 3 * kMaxN;
  double* dinv = A.scratch + 4 * kMaxN;
  const double lam = A.lam, c = A.c, d = A.d, e = d - c * c;

  // Jacobi diagonal: lam((L^2)_ii + 2c L_ii + d) + omega_i;  x0 = 0, r0 = b
  double v1[1] = {0.0};
  for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
    const int i = beg + li;
    double l2 = 0.0, li_ii = 0.0;
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      l2 += A.val[q] * A.val[q];
      if (A.col[q] == i) li_ii += A.val[q];
    }
    const double dd = lam * (l2 + 2.0 * c * li_ii + d) + A.omega[i];
    dinv[i] = dd > 0.0 ? 1.0 / dd : 1.0;
    A.x[i] = 0.0;
    const double bi = A.b[i];
    r[i] = bi;
    v1[0] += bi * bi;
  }
  na_block_sum<1>(v1, scr, red);
  cl.sync();
  na_cluster_sum<1>(cl, red, scal, C);
  const double bb = scal[0];
  int it = 0, status = 0;
  double rho = 0.0;
  if (bb > 0.0) {
    const double tol2 = A.tol * A.tol * bb;
    double gam_prev = 1.0, alpha_prev = 1.0;
    int cur = 0;
    for (;;) {
      double* ub = cur ? ub1 : ub0;
      for (int li = threadIdx.x; li < nloc; li += blockDim.x) ub[li] = r[beg + li] * dinv[beg + li];
      cl.sync();
      for (int li = threadIdx.x; li < nloc; li += blockDim.x) tb[li] = na_row(A, beg + li, c, ub, cl);
      cl.sync();
      double v[3] = {0.0, 0.0, 0.0};
      for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
        const int i = beg + li;
        const double ui = ub[li];
        const double wi = lam * (na_row(A, i, c, tb, cl) + e * ui) + A.omega[i] * ui;
        const double ri = r[i];
        w[i] = wi;
        v[0] += ri * ui;
        v[1] += ui * wi;
        v[2] += ri * ri;
      }
      na_block_sum<3>(v, scr, red);
      cl.sync();
      na_cluster_sum<3>(cl, red, scal, C);
      const double gam = scal[0], del = scal[1];
      rho = scal[2];
      if (rho <= tol2) break;
      if (it >= A.maxit) {
        status = 1;
        break;
      }
      double beta = 0.0, den = del;
      if (it > 0) {
        beta = gam / gam_prev;
        den = del - beta * gam / alpha_prev;
      }
      if (!(den > 0.0) || !isfinite(den)) {
        status = 2;
        break;
      }
      const double alpha = gam / den;
      for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
        const int i = beg + li;
        const double pi = it == 0 ? ub[li] : ub[li] + beta * p[i];
        const double si = it == 0 ? w[i] : w[i] + beta * s[i];
        p[i] = pi;
        s[i] = si;
        A.x[i] += alpha * pi;
        r[i] -= alpha * si;
      }
      gam_prev = gam;
      alpha_prev = alpha;
      cur ^= 1;
      ++it;
    }
  }
  cl.sync();  // no CTA leaves while another may read its shared memory
  if (rank == 0 && threadIdx.x == 0) {
    double* st = A.scratch + kStatOff;
    st[0] = (double)it;
    st[1] = (double)status;
    st[2] = bb > 0.0 ? sqrt(rho / bb) : 0.0;
    st[3] = 1.0;  // written: the kernel ran to completion
  }
}

size_t na_smem(int chunk) { return sizeof(double) * (3 * (size_t)chunk + 8 + 128 + 8); }

// With the device current: the device address of the scratch array in the
// current context and the kernel's launch attributes.  Looked up on every call,
// so nothing cached can outlive a context reset.
cr_status na_setup(double** out, std::string& err) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess || !ptr) {
    err = std::string("cudaGetSymbolAddress(scratch) failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return CR_ECUDA;
  }
  e = cudaFuncSetAttribute(na_pcg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(na_pcg_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    err = std::string("kernel attribute set-up failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return CR_ECUDA;
  }
  *out = static_cast<double*>(ptr);
  return CR_OK;
}

bool na_cluster_ok(int cs, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, na_pcg_kernel, &cfg) != cudaSuccess || ncl < 1) {
    cudaGetLastError();
    return false;
  }
  return true;
}

}  // namespace

extern "C" cr_status cr_solve_u_noalloc(int64_t n, const int32_t* rowptr_dev, const int32_t* col_dev,
                                        const double* val_dev, double lambda, double c, double d,
                                        const double* omega_dev, const double* rhs_dev, double* u_hat_dev, double tol,
                                        int32_t maxit, int32_t* iters, void* stream) {
  auto bad = [](cr_status s, const std::string& m) {
    cr::set_global_error(m);
    return s;
  };
  if (n < 1 || n > kMaxN)
    return bad(CR_EINVAL, "cr_solve_u_noalloc: n = " + std::to_string(n) + " outside [1, " + std::to_string(kMaxN) +
                              "], the size of its static scratch");
  if (!rowptr_dev || !col_dev || !val_dev || !omega_dev || !rhs_dev || !u_hat_dev)
    return bad(CR_EINVAL, "cr_solve_u_noalloc: null pointer");
  if (!(tol > 0.0) || maxit < 1 || !(lambda > 0.0) || !std::isfinite(c) || !std::isfinite(d))
    return bad(CR_EINVAL, "cr_solve_u_noalloc: bad tol, maxit, lambda, c or d");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return bad(CR_ECUDA, "cr_solve_u_noalloc: no current CUDA device");
  }
  std::string err;
  double* scratch = nullptr;
  cr_status s = na_setup(&scratch, err);
  if (s != CR_OK) return bad(s, err);
  const int ni = (int)n;
  int desired = std::min(16, std::max(1, (ni + 479) / 480));
  int cs = 0, chunk = 0;
  for (int c2 = desired; c2 >= 1; --c2) {
    const int ch = (ni + c2 - 1) / c2;
    if (na_smem(ch) > 227 * 1024) break;
    if (na_cluster_ok(c2, na_smem(ch))) {
      cs = c2;
      chunk = ch;
      break;
    }
  }
  if (cs == 0) return bad(CR_EINVAL, "cr_solve_u_noalloc: no feasible cluster for n = " + std::to_string(n));
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(scratch + kStatOff, 0, 8 * sizeof(double), st) != cudaSuccess) {
    cudaGetLastError();
    return bad(CR_ECUDA, "cr_solve_u_noalloc: clearing the status words failed");
  }
  NaArgs a{};
  a.n = ni;
  a.rp = rowptr_dev;
  a.col = col_dev;
  a.val = val_dev;
  a.lam = lambda;
  a.c = c;
  a.d = d;
  a.omega = omega_dev;
  a.b = rhs_dev;
  a.x = u_hat_dev;
  a.scratch = scratch;
  a.tol = tol;
  a.maxit = maxit;
  a.chunk = chunk;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = na_smem(chunk);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cr::count_launch();
  cudaError_t e = cudaLaunchKernelEx(&cfg, na_pcg_kernel, a);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bad(CR_ECUDA, std::string("cr_solve_u_noalloc: launch failed: ") + cudaGetErrorString(e));
  }
  double hst[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(hst, scratch + kStatOff, sizeof(hst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bad(CR_ECUDA, std::string("cr_solve_u_noalloc: ") + cudaGetErrorString(e));
  }
  if (iters) *iters = (int32_t)hst[0];
  if (hst[3] != 1.0) return bad(CR_ECUDA, "cr_solve_u_noalloc: kernel did not complete");
  if (hst[1] == 2.0) return bad(CR_ENOTCONV, "cr_solve_u_noalloc: PCG breakdown");
  if (hst[1] == 1.0) return bad(CR_ENOTCONV, "cr_solve_u_noalloc: PCG reached maxit");
  return CR_OK;
}
