// Grid-wide Jacobi PCG for the ALS sub-systems (Eq. ALS_linsys, u side;
// Eq. ALS_linsys_v, v side) on voxel grids too large for one thread-block
// cluster's shared memory.  Vectors stream from HBM; every SM takes part.
//
// One persistent cooperative launch runs the whole solve.  Block b owns the
// contiguous rows [b*chunk, (b+1)*chunk).  Each PCG iteration is three
// sweeps separated by a bounded grid barrier (the v side adds one short
// sweep: block a adds column a of the per-block partial X^T p, so that every
// block then reads y = s o X^T p for its data term X diag(s) X^T p):
//   A2a  p = D^-1 r + beta p_old and t = (L + cI) p.  Row i needs p on its
//        one-hop neighbourhood, recomputed from r and p_old (p is double
//        buffered), so no barrier separates the p update from the stencil;
//   A2b  q = lam ((L + cI) t + e p) + data(p), and the block's partial <p, q>;
//   B    alpha = rho / <p, q>, x += alpha p, r -= alpha q, and the partials
//        of rho' = <r, D^-1 r> and |r|^2.
// The operator holds (L + cI)^2; splitting it through t keeps every row's
// loads one hop deep, with the neighbour indices fetched before the values.
// Reads of data that other blocks wrote before the last grid barrier are
// ordinary (L1-cached) loads: the barrier's acquire fence at GPU scope, taken
// before the block passes its CTA barrier, makes those writes visible (the
// cooperative-groups grid synchronisation pattern), and adjacent rows share
// most of their neighbourhoods in L1.
// Every block adds the per-block partial sums itself, in one fixed order, so
// all blocks hold bit-identical scalars and take identical decisions.
// T = float: float32 vectors and arithmetic with double-float (two-float)
// accumulation of the inner products; T = double: float64 throughout (on
// GB300 the float64 form is bound by float64 arithmetic, not by HBM).
// Bytes per row and iteration in float32 (unit-weight Laplacian, K = 6):
// A2a reads r, p_old, D^-1, L_ii, the neighbour table and writes p, t (48 B);
// A2b reads t, p, L_ii, omega, the table and writes q (44 B); B reads x, p, r,
// q, D^-1 and writes x, r (28 B): 120 B, against the 64 B of the two-sweep
// minimum (r, x, p, q once each way, D^-1, omega, the table): the table and
// L_ii are read twice and t makes one round trip.
#include <algorithm>

#include "cr_common.cuh"
#include "cr_df.cuh"

namespace cr {

namespace {

constexpr int kGThreads = 512;
constexpr long long kGridSpin = 1ll << 24;

struct GridPcg {
  DevLap L;
  double lam;
  const double* coef;  // device [2]: c, d of the shifted operator
  int side;            // 0: u side (omega data term), 1: v side (X diag(s) X^T)
  int m;
  const double* s;     // v side [m]
  const int* xr_ptr;   // v side: X by rows (CSR)
  const int* xr_col;
  const double* xr_val;
  const int* xc_ptr;   // v side: X by columns (CSC, rows ascending)
  const int* xc_row;
  const double* xc_val;
  const double* b;     // [n] right side (float64)
  double* x;           // [n] in: x0, out: solution (float64)
  const double* dinv64;  // [n] Jacobi inverse diagonal (float64)
  const double* omt64;   // [n] u side omega (float64)
  void* xs;            // [n] T work: x
  void* rs;            // [n] T: r
  void* p0;            // [n] T: p, two buffers (old / new)
  void* p1;
  void* qs;            // [n] T: q = A_hat p
  void* ts;            // [n] T: t = (L + cI) p
  void* ds;            // [n] T: D^-1
  void* os;            // [n] T: omega (u side)
  void* gs;            // [n] T: L_ii
  double* part;        // [nb * kParts] per-block partial sums
  double* ypart;       // v side [nb * m] per-block partial X^T p
  double* yglob;       // v side [m] y = s o X^T p
  unsigned* bar;       // [2] barrier counter, generation
  int* err;            // barrier timeout flag
  int nb, chunk;
  double tol;
  int maxit;
  PcgStat* stat;
};

constexpr int kParts = 4;  // (p,q), rho, |r|^2, |b|^2

__device__ __forceinline__ bool grid_sync(const GridPcg& a) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
    int good = 1;
    if (arrived == (unsigned)a.nb) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (*(volatile int*)a.err) {
          good = 0;
          break;
        }
        if (++spins > kGridSpin) {
          atomicExch(a.err, 1);
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok = good && !*(volatile int*)a.err;
  }
  __syncthreads();
  return ok;
}

// Accumulator of an inner product: double-float for float32 vectors, double otherwise.
template <class T>
struct Acc;
template <>
struct Acc<float> {
  DF v{0.f, 0.f};
  __device__ void add(float a, float b) { v = df_add(v, df_prod(a, b)); }
  __device__ double get() const { return (double)v.hi + (double)v.lo; }
};
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ double get() const { return v; }
};

// Block sum of NV doubles in a fixed tree order; result in out[] of thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* out) {
  __shared__ double sh[kGThreads / 32][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[w][k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int q = 0; q < kGThreads / 32; ++q) t += sh[q][k];
      out[k] = t;
    }
  }
  __syncthreads();
}

// Sum of part[b * stride + k] over all blocks b, in the same order in every block.
__device__ __forceinline__ double sum_parts(const double* part, int nb, int stride, int k) {
  __shared__ double sh[kGThreads / 32];
  __shared__ double res;
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(part + (size_t)b * stride + k);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) sh[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int q = 0; q < kGThreads / 32; ++q) u += sh[q];
    res = u;
  }
  __syncthreads();
  const double out = res;
  __syncthreads();
  return out;
}

// Neighbour indices of row i (KM slots; -1 = none).  The table is never
// written during the solve: read-only path.
template <int KM>
__device__ __forceinline__ void load_nbrs(const DevLap& L, int i, int (&q)[KM]) {
#pragma unroll
  for (int sl = 0; sl < KM; ++sl) q[sl] = sl < L.K ? __ldg(L.nbr + (size_t)sl * L.n + i) : -1;
}

// Row i of (L + cI) v with the neighbour indices already loaded; v(l) from the functor.
template <class T, int KM, class VF>
__device__ __forceinline__ T shifted_row(const DevLap& L, const T* gs, int i, const int (&q)[KM], T c,
                                         const VF& v) {
  T acc = (gs[i] + c) * v(i);
#pragma unroll
  for (int sl = 0; sl < KM; ++sl) {
    if (q[sl] >= 0) {
      const T w = L.offw ? (T)__ldg(L.offw + (size_t)sl * L.n + i) : (T)-1;
      acc = fma(w, v(q[sl]), acc);
    }
  }
  return acc;
}

// f(i, q) over the block's rows, two rows per thread and step: both rows'
// neighbour indices are loaded before either row's values, so each thread
// keeps two rows' loads in flight (the sweeps are bound by memory latency).
template <int KM, class F>
__device__ __forceinline__ void for_rows2(const DevLap& L, int lo, int hi, const F& f) {
  const int bd = blockDim.x;
  for (int i0 = lo + threadIdx.x; i0 < hi; i0 += 2 * bd) {
    const int i1 = i0 + bd;
    int q0[KM], q1[KM];
    load_nbrs<KM>(L, i0, q0);
    if (i1 < hi) load_nbrs<KM>(L, i1, q1);
    f(i0, q0);
    if (i1 < hi) f(i1, q1);
  }
}

// Column sums of X restricted to rows [lo, hi): out[a] = sum_i X_ia v_i, one
// warp per column, the column's row range found by binary search (rows of a
// CSC column ascend), lanes summed in a fixed order.
template <class T>
__device__ __forceinline__ void xt_partial(const GridPcg& a, int lo, int hi, const T* v, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int col = w; col < a.m; col += nw) {
    int b0 = a.xc_ptr[col], b1 = a.xc_ptr[col + 1];
    // first entry with row >= lo
    int l = b0, h = b1;
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (a.xc_row[mid] < lo) l = mid + 1; else h = mid;
    }
    const int s0 = l;
    h = b1;
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (a.xc_row[mid] < hi) l = mid + 1; else h = mid;
    }
    const int s1 = l;
    double t = 0.0;
    for (int q = s0 + lane; q < s1; q += 32) t = fma(a.xc_val[q], (double)v[a.xc_row[q]], t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) out[col] = t;
  }
}

// Second stage of the v side's X^T v: block a adds column a of the per-block
// partials (fixed order) and stores y_a = s_a (X^T v)_a.
__device__ __forceinline__ void reduce_y_global(const GridPcg& a) {
  __shared__ double sh[kGThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int col = blockIdx.x; col < a.m; col += a.nb) {
    double t = 0.0;
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) t += __ldcg(a.ypart + (size_t)b * a.m + col);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int q = 0; q < kGThreads / 32; ++q) u += sh[q];
      a.yglob[col] = a.s[col] * u;
    }
    __syncthreads();
  }
}

// y into shared memory for the block's data-term rows
__device__ __forceinline__ void load_y(const GridPcg& a, double* ys) {
  for (int col = threadIdx.x; col < a.m; col += blockDim.x) ys[col] = __ldcg(a.yglob + col);
  __syncthreads();
}

// Data term of row i: omega_i v_i (u side) or sum_a X_ia y_a (v side, y in shared memory).
template <class T>
__device__ __forceinline__ T data_row(const GridPcg& a, const T* om, const double* ys, int i, T vi) {
  if (a.side == 0) return om[i] * vi;
  T acc = (T)0;
  for (int q = a.xr_ptr[i]; q < a.xr_ptr[i + 1]; ++q) acc = fma((T)a.xr_val[q], (T)ys[a.xr_col[q]], acc);
  return acc;
}

template <class T, int KM>
__global__ void __launch_bounds__(kGThreads) pcg_grid_kernel(const GridPcg a) {
  extern __shared__ double ys[];  // v side: y = s o (X^T v), m entries
  __shared__ double red[kParts];
  T* xs = (T*)a.xs;
  T* rs = (T*)a.rs;
  T* qs = (T*)a.qs;
  T* ts = (T*)a.ts;
  T* dv = (T*)a.ds;
  T* om = (T*)a.os;
  T* gs = (T*)a.gs;
  const int n = a.L.n;
  const int lo = min(n, blockIdx.x * a.chunk), hi = min(n, lo + a.chunk);
  const double cd = a.coef[0], dd = a.coef[1];
  const T c = (T)cd, e = (T)(dd - cd * cd), lam = (T)a.lam;
  int it = 0, status = 0;
  double rho = 0.0, rr = 0.0, bb = 0.0;

  // ---- set-up: T copies of x0, D^-1, omega, L_ii
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    xs[i] = (T)a.x[i];
    dv[i] = (T)a.dinv64[i];
    gs[i] = (T)a.L.diag[i];
    if (a.side == 0) om[i] = (T)a.omt64[i];
  }
  if (!grid_sync(a)) goto done;
  // ---- t = (L + cI) x0; v side partial X^T x0
  {
    auto xv = [&](int l) { return xs[l]; };
    for_rows2<KM>(a.L, lo, hi, [&](int i, const int (&q)[KM]) { ts[i] = shifted_row<T, KM>(a.L, gs, i, q, c, xv); });
  }
  if (a.side == 1) xt_partial<T>(a, lo, hi, xs, a.ypart + (size_t)blockIdx.x * a.m);
  if (!grid_sync(a)) goto done;
  if (a.side == 1) {
    reduce_y_global(a);
    if (!grid_sync(a)) goto done;
    load_y(a, ys);
  }
  // ---- r0 = b - A_hat x0; partial rho, |r|^2, |b|^2
  {
    auto tv = [&](int l) { return ts[l]; };
    Acc<T> a_rho, a_rr, a_bb;
    for_rows2<KM>(a.L, lo, hi, [&](int i, const int (&q)[KM]) {
      const T xi = xs[i];
      const T bi = (T)a.b[i];
      const T ri = bi - (lam * (shifted_row<T, KM>(a.L, gs, i, q, c, tv) + e * xi) + data_row<T>(a, om, ys, i, xi));
      rs[i] = ri;
      a_rho.add(ri, dv[i] * ri);
      a_rr.add(ri, ri);
      a_bb.add(bi, bi);
    });
    double v[3] = {a_rho.get(), a_rr.get(), a_bb.get()};
    block_reduce<3>(v, red);
    if (threadIdx.x == 0) {
      double* pb = a.part + (size_t)blockIdx.x * kParts;
      pb[1] = red[0];
      pb[2] = red[1];
      pb[3] = red[2];
    }
  }
  if (!grid_sync(a)) goto done;
  rho = sum_parts(a.part, a.nb, kParts, 1);
  rr = sum_parts(a.part, a.nb, kParts, 2);
  bb = sum_parts(a.part, a.nb, kParts, 3);
  if (bb > 0.0) {
    const double tol2 = a.tol * a.tol * bb;
    double rho_prev = 1.0;
    for (;;) {
      if (rr <= tol2) break;
      if (it >= a.maxit) {
        status = 1;
        break;
      }
      T* pold = (T*)((it & 1) ? a.p1 : a.p0);
      T* pnew = (T*)((it & 1) ? a.p0 : a.p1);
      // ---- sweep A2a: p = D^-1 r + beta p_old (recomputed on the one-hop
      //      neighbourhood), t = (L + cI) p; v side partial X^T p
      {
        const bool first = it == 0;
        const T beta = (T)(first ? 0.0 : rho / rho_prev);
        auto pn = [&](int l) -> T {
          const T z = dv[l] * rs[l];
          return first ? z : fma(beta, pold[l], z);
        };
        for_rows2<KM>(a.L, lo, hi, [&](int i, const int (&q)[KM]) {
          ts[i] = shifted_row<T, KM>(a.L, gs, i, q, c, pn);
          pnew[i] = pn(i);
        });
      }
      if (a.side == 1) {
        __syncthreads();
        xt_partial<T>(a, lo, hi, pnew, a.ypart + (size_t)blockIdx.x * a.m);
      }
      if (!grid_sync(a)) goto done;
      if (a.side == 1) {
        reduce_y_global(a);
        if (!grid_sync(a)) goto done;
        load_y(a, ys);
      }
      // ---- sweep A2b: q = lam ((L + cI) t + e p) + data(p); partial <p, q>
      {
        auto tv = [&](int l) { return ts[l]; };
        Acc<T> a_pq;
        for_rows2<KM>(a.L, lo, hi, [&](int i, const int (&q)[KM]) {
          const T pi = pnew[i];
          const T qi = lam * (shifted_row<T, KM>(a.L, gs, i, q, c, tv) + e * pi) + data_row<T>(a, om, ys, i, pi);
          qs[i] = qi;
          a_pq.add(pi, qi);
        });
        double v[1] = {a_pq.get()};
        block_reduce<1>(v, red);
        if (threadIdx.x == 0) a.part[(size_t)blockIdx.x * kParts + 0] = red[0];
      }
      if (!grid_sync(a)) goto done;
      const double pq = sum_parts(a.part, a.nb, kParts, 0);
      if (!(pq > 0.0)) {
        status = 2;
        break;
      }
      // ---- sweep B: x += alpha p, r -= alpha q; partial rho, |r|^2
      {
        const T alpha = (T)(rho / pq);
        Acc<T> a_rho, a_rr;
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
          xs[i] = fma(alpha, pnew[i], xs[i]);
          const T ri = fma(-alpha, qs[i], rs[i]);
          rs[i] = ri;
          a_rho.add(ri, dv[i] * ri);
          a_rr.add(ri, ri);
        }
        double v[2] = {a_rho.get(), a_rr.get()};
        block_reduce<2>(v, red);
        if (threadIdx.x == 0) {
          double* pb = a.part + (size_t)blockIdx.x * kParts;
          pb[1] = red[0];
          pb[2] = red[1];
        }
      }
      ++it;
      if (!grid_sync(a)) goto done;
      rho_prev = rho;
      rho = sum_parts(a.part, a.nb, kParts, 1);
      rr = sum_parts(a.part, a.nb, kParts, 2);
    }
  }
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) a.x[i] = (double)xs[i];
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PcgStat st;
    st.iters = it;
    st.status = *(volatile int*)a.err ? 3 : status;
    st.relres = bb > 0.0 ? sqrt(fmax(rr, 0.0) / bb) : 0.0;
    st.bnorm = sqrt(bb);
    *a.stat = st;
  }
}

}  // namespace
}  // namespace cr

namespace cr {

// Largest block count that is co-resident for the kernel variant (float32 or
// float64; 6 or up to kMaxSlots neighbour slots), at most two blocks of
// kGThreads per SM (cooperative launch); 0 if it cannot run.
const void* grid_kernel_fn(bool fp32, int K) {
  const bool k6 = K <= 6;
  return fp32 ? (k6 ? (const void*)pcg_grid_kernel<float, 6> : (const void*)pcg_grid_kernel<float, kMaxSlots>)
              : (k6 ? (const void*)pcg_grid_kernel<double, 6> : (const void*)pcg_grid_kernel<double, kMaxSlots>);
}

int pcg_grid_blocks(bool fp32, int m, int K) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(double) * (size_t)std::max(m, 1);
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grid_kernel_fn(fp32, K), kGThreads, smem);
  if (e != cudaSuccess || per < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms * std::min(per, 2);
}

size_t pcg_grid_work_elems(int n) { return (size_t)9 * n; }

cudaError_t pcg_grid_launch(const PcgArgs& a, int side, const int* xc_ptr, const int* xc_row, const double* xc_val,
                            double* work, double* part, double* ypart, double* yglob, unsigned* bar, int* err,
                            int nb, cudaStream_t st) {
  const int n = a.L.n;
  if (nb < 1 || n < 1) return cudaErrorInvalidValue;
  GridPcg g{};
  g.L = a.L;
  g.lam = a.lam;
  g.coef = a.coef;
  g.side = side;
  g.m = a.m;
  g.s = a.s;
  g.xr_ptr = a.X.xr_ptr;
  g.xr_col = a.X.xr_col;
  g.xr_val = a.X.xr_val;
  g.xc_ptr = xc_ptr;
  g.xc_row = xc_row;
  g.xc_val = xc_val;
  g.b = a.b;
  g.x = a.x;
  g.dinv64 = a.dinv;
  g.omt64 = a.omt;
  const size_t word = a.fp32 ? sizeof(float) : sizeof(double);
  char* w = reinterpret_cast<char*>(work);
  void** slots[9] = {&g.xs, &g.rs, &g.p0, &g.p1, &g.qs, &g.ts, &g.ds, &g.os, &g.gs};
  for (int k = 0; k < 9; ++k) *slots[k] = w + (size_t)k * n * word;
  g.part = part;
  g.ypart = ypart;
  g.yglob = yglob;
  g.bar = bar;
  g.err = err;
  g.nb = nb;
  g.chunk = (n + nb - 1) / nb;
  g.tol = a.tol;
  g.maxit = a.maxit;
  g.stat = a.stat;
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  void* args[] = {&g};
  const size_t smem = sizeof(double) * (size_t)std::max(a.m, 1);
  count_launch();
  return cudaLaunchCooperativeKernel(grid_kernel_fn(a.fp32 != 0, a.L.K), dim3(nb), dim3(kGThreads), args, smem, st);
}

}  // namespace cr
