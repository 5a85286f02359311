// Float64 dense and sparse building blocks of the greedy solver: panel
// products for the residual products R_j v / R_j^T u, Gram-Schmidt, the
// projected coefficient matrices and the Galerkin CG of Eq. (Proj_Sylv).
//
// Every reduction has a fixed order (no atomics), so results are bitwise
// reproducible.  GB300's float64 rate is low (about 2 FMA per SM per clock),
// so the kernels spread even small products over many CTAs: the generic GEMM
// uses 16x16 output tiles and splits the reduction dimension until a few
// hundred CTAs are busy, adding the split partial sums in order.
#include <cstdio>

#include "cr_common.cuh"

namespace cr {

std::atomic<long long> g_launches{0};

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr int TB = 16;

__global__ void gemm_kernel(int M, int N, int K, MatView A, MatView B, int kchunk, double alpha, double beta,
                            double* __restrict__ C, int64_t sci, int64_t scl, double* __restrict__ part) {
  __shared__ double As[TB][TB + 1];  // [k][i]
  __shared__ double Bs[TB][TB + 1];  // [k][l]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * TB, l0 = blockIdx.y * TB;
  const int s = blockIdx.z;
  const int k0 = s * kchunk, k1 = min(K, k0 + kchunk);
  const bool a_unit_i = A.si == 1;
  const bool b_unit_k = B.si == 1;  // B(k, l): k is B's "i" index
  double acc = 0.0;
  for (int kk = k0; kk < k1; kk += TB) {
    {
      const int iq = a_unit_i ? tx : ty, kq = a_unit_i ? ty : tx;
      const int i = i0 + iq, k = kk + kq;
      As[kq][iq] = (i < M && k < k1) ? A.ptr[(int64_t)i * A.si + (int64_t)k * A.sk] : 0.0;
    }
    {
      const int kq = b_unit_k ? tx : ty, lq = b_unit_k ? ty : tx;
      const int k = kk + kq, l = l0 + lq;
      Bs[kq][lq] = (k < k1 && l < N) ? B.ptr[(int64_t)k * B.si + (int64_t)l * B.sk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TB; ++q) acc = fma(As[q][ty], Bs[q][tx], acc);
    __syncthreads();
  }
  const int i = i0 + ty, l = l0 + tx;
  if (i >= M || l >= N) return;
  if (part) {
    part[((int64_t)s * M + i) * N + l] = acc;
  } else {
    double* c = C + (int64_t)i * sci + (int64_t)l * scl;
    *c = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *c);
  }
}

__global__ void gemm_reduce_kernel(int M, int N, int S, const double* __restrict__ part, double alpha, double beta,
                                   double* __restrict__ C, int64_t sci, int64_t scl) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * N) return;
  const int i = (int)(t / N), l = (int)(t % N);
  double acc = 0.0;
  for (int s = 0; s < S; ++s) acc += part[((int64_t)s * M + i) * N + l];
  double* c = C + (int64_t)i * sci + (int64_t)l * scl;
  *c = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *c);
}

// one warp per output column p
// out[p] = alpha * A(:, p)^T w (+ beta out[p]): one CTA of 256 threads per column,
// four independent accumulators per thread (rows strided by 256, so loads of
// consecutive threads coalesce and four are in flight), then a fixed-order
// reduction over the CTA (warp shuffles, then the eight warp sums in order).
constexpr int kGvThreads = 256;

__global__ void __launch_bounds__(kGvThreads) gemv_t_kernel(int n, int k, const double* __restrict__ A, int64_t lda,
                                                            const double* __restrict__ w, double* out,
                                                            int64_t ostride, double alpha, double beta) {
  const int p = blockIdx.x;
  if (p >= k) return;
  const double* a = A + (int64_t)p * lda;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int i = threadIdx.x;
  for (; i + 3 * kGvThreads < n; i += 4 * kGvThreads) {
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = fma(a[i + u * kGvThreads], w[i + u * kGvThreads], acc[u]);
  }
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int ii = i + u * kGvThreads;
    if (ii < n) acc[u] = fma(a[ii], w[ii], acc[u]);
  }
  double v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  v = warp_sum(v);
  __shared__ double red[kGvThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kGvThreads / 32; ++q) t += red[q];
    double* o = out + (int64_t)p * ostride;
    *o = beta == 0.0 ? alpha * t : fma(alpha, t, beta * *o);
  }
}

// y[i] = alpha * sum_p A(i, p) c[p] (+ beta y[i]): a CTA takes 32 consecutive rows;
// its eight warps split the columns in eight fixed ranges (lane = row, so loads
// coalesce), four accumulators per thread, and the eight partial sums of a row
// are added in order.
__global__ void __launch_bounds__(kGvThreads) gemv_n_kernel(int n, int k, const double* __restrict__ A, int64_t lda,
                                                            const double* __restrict__ c, int64_t cs, double* y,
                                                            double alpha, double beta) {
  extern __shared__ double cs_sm[];
  for (int p = threadIdx.x; p < k; p += blockDim.x) cs_sm[p] = c[(int64_t)p * cs];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int kc = (k + 7) / 8, p0 = min(k, wid * kc), p1 = min(k, p0 + kc);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    const double* a = A + i;
    int p = p0;
    for (; p + 3 < p1; p += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(a[(int64_t)(p + u) * lda], cs_sm[p + u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (p + u < p1) acc[u] = fma(a[(int64_t)(p + u) * lda], cs_sm[p + u], acc[u]);
  }
  __shared__ double part[8][33];
  part[wid][lane] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  __syncthreads();
  if (wid == 0 && i < n) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    y[i] = beta == 0.0 ? alpha * t : fma(alpha, t, beta * y[i]);
  }
}

__global__ void dot_kernel(int n, const double* __restrict__ x, const double* __restrict__ y, double* out) {
  __shared__ double scr[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(x[i], y[i], acc);
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) scr[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? scr[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) *out = t;
  }
}

__global__ void spmv_xt_kernel(int m, const int* __restrict__ cp, const int* __restrict__ row,
                               const double* __restrict__ val, const double* __restrict__ v, double* out,
                               int64_t ostride) {
  const int lane = threadIdx.x & 31;
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (a >= m) return;
  double acc = 0.0;
  for (int p = cp[a] + lane; p < cp[a + 1]; p += 32) acc = fma(val[p], v[row[p]], acc);
  acc = warp_sum(acc);
  if (lane == 0) out[(int64_t)a * ostride] = acc;
}

__global__ void spmv_x_kernel(int n, const int* __restrict__ rp, const int* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ c, double* y, double alpha,
                              double beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(val[p], c[col[p]], acc);
  y[i] = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * y[i]);
}

// out[a] = sum_i Om(i, a) u_i^2: one CTA per injection, laid out as gemv_t_kernel.
__global__ void __launch_bounds__(kGvThreads) omega_sq_kernel(int n, int m, const uint8_t* __restrict__ Om,
                                                              int64_t ldo, const double* __restrict__ u,
                                                              double* out) {
  const int a = blockIdx.x;
  if (a >= m) return;
  const uint8_t* o = Om + (int64_t)a * ldo;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int i = threadIdx.x;
  for (; i + 3 * kGvThreads < n; i += 4 * kGvThreads) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double x = u[i + q * kGvThreads];
      acc[q] = fma((double)o[i + q * kGvThreads] * x, x, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int ii = i + q * kGvThreads;
    if (ii < n) acc[q] = fma((double)o[ii] * u[ii], u[ii], acc[q]);
  }
  double v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  v = warp_sum(v);
  __shared__ double red[kGvThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kGvThreads / 32; ++q) t += red[q];
    out[a] = t;
  }
}

__global__ void scale_inv_norm_kernel(int n, const double* __restrict__ x, const double* nrm2, double* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = x[i] / sqrt(*nrm2);
}

__global__ void copy_kernel(int n, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i];
}

__global__ void fill_kernel(int64_t n, double v, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}

// out[i + a*ldo] = sum_q G_a[i + q*ldg] * w[q + a*ldw]; block = (row tile, a)
__global__ void batched_gemv_kernel(int j, const double* __restrict__ G, int64_t ldg, int64_t gstride,
                                    const double* __restrict__ w, int64_t ldw, double* __restrict__ out,
                                    int64_t ldo) {
  extern __shared__ double wsm[];
  const int a = blockIdx.y;
  for (int q = threadIdx.x; q < j; q += blockDim.x) wsm[q] = w[q + (int64_t)a * ldw];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= j) return;
  const double* g = G + (int64_t)a * gstride;
  double acc = 0.0;
  for (int q = 0; q < j; ++q) acc = fma(g[i + (int64_t)q * ldg], wsm[q], acc);
  out[i + (int64_t)a * ldo] = acc;
}

}  // namespace

void gemm(int M, int N, int K, double alpha, MatView A, MatView B, double beta, double* C, int64_t sci,
          int64_t scl, double* ws, size_t ws_elems, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    // C = beta * C: the reduce kernel with no partial sums
    if (beta == 1.0) return;
    const int64_t tot = (int64_t)M * N;
    count_launch();
    gemm_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, 0, ws, 0.0, beta, C, sci, scl);
    return;
  }
  const int tiles = ((M + TB - 1) / TB) * ((N + TB - 1) / TB);
  int S = (2 * 152 + tiles - 1) / tiles;
  const int smax = (K + 63) / 64;
  if (S > smax) S = smax;
  if (S < 1) S = 1;
  while (S > 1 && (size_t)S * M * N > ws_elems) --S;
  int kchunk = (K + S - 1) / S;
  kchunk = ((kchunk + TB - 1) / TB) * TB;
  S = (K + kchunk - 1) / kchunk;
  dim3 grid((M + TB - 1) / TB, (N + TB - 1) / TB, S);
  dim3 blk(TB, TB);
  if (S == 1) {
    count_launch();
    gemm_kernel<<<grid, blk, 0, st>>>(M, N, K, A, B, kchunk, alpha, beta, C, sci, scl, nullptr);
  } else {
    count_launch();
    gemm_kernel<<<grid, blk, 0, st>>>(M, N, K, A, B, kchunk, 1.0, 0.0, C, sci, scl, ws);
    const int64_t tot = (int64_t)M * N;
    count_launch();
    gemm_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, S, ws, alpha, beta, C, sci, scl);
  }
}

void gemv_t(int n, int k, const double* A, int64_t lda, const double* w, double* out, int64_t ostride,
            double alpha, double beta, cudaStream_t st) {
  if (k <= 0) return;
  count_launch();
  gemv_t_kernel<<<k, kGvThreads, 0, st>>>(n, k, A, lda, w, out, ostride, alpha, beta);
}

void gemv_n(int n, int k, const double* A, int64_t lda, const double* c, int64_t cstride, double* y, double alpha,
            double beta, cudaStream_t st) {
  if (n <= 0) return;
  if (k <= 0) {
    if (beta == 1.0) return;
    count_launch();
    gemv_n_kernel<<<(n + 31) / 32, kGvThreads, 0, st>>>(n, 0, A, lda, c, cstride, y, alpha, beta);
    return;
  }
  count_launch();
  gemv_n_kernel<<<(n + 31) / 32, kGvThreads, sizeof(double) * k, st>>>(n, k, A, lda, c, cstride, y, alpha, beta);
}

void dot(int n, const double* x, const double* y, double* out, cudaStream_t st) {
  count_launch();
  dot_kernel<<<1, 1024, 0, st>>>(n, x, y, out);
}

void spmv_xt(int m, const int* colptr, const int* row, const double* val, const double* v, double* out,
             int64_t ostride, cudaStream_t st) {
  if (m <= 0) return;
  count_launch();
  spmv_xt_kernel<<<(m + 7) / 8, 256, 0, st>>>(m, colptr, row, val, v, out, ostride);
}

void spmv_x(int n, const int* rowptr, const int* col, const double* val, const double* c, double* y, double alpha,
            double beta, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  spmv_x_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, col, val, c, y, alpha, beta);
}

void omega_sq_dots(int n, int m, const uint8_t* Om, int64_t ldo, const double* u, double* out, cudaStream_t st) {
  if (m <= 0) return;
  count_launch();
  omega_sq_kernel<<<m, kGvThreads, 0, st>>>(n, m, Om, ldo, u, out);
}

void scale_by_inv_norm(int n, const double* x, const double* nrm2, double* y, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  scale_inv_norm_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, x, nrm2, y);
}

void copy(int n, const double* x, double* y, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  copy_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, x, y);
}

void fill(int64_t n, double v, double* y, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, v, y);
}

void batched_gemv(int j, int m, const double* G, int64_t ldg, int64_t gstride, const double* w, int64_t ldw,
                  double* out, int64_t ldo, cudaStream_t st) {
  if (j <= 0 || m <= 0) return;
  dim3 grid((j + 127) / 128, m);
  count_launch();
  batched_gemv_kernel<<<grid, 128, sizeof(double) * j, st>>>(j, G, ldg, gstride, w, ldw, out, ldo);
}

}  // namespace cr
