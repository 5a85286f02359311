// Small kernels of the greedy driver: coefficient vectors of the residual
// products, symmetric borders of the projected matrices, the masked data
// residual E = Omega o (Y - U Z V^T X), Galerkin CG updates and the core
// matrix of the residual norm.  All reductions are fixed-order.
#include "cr_common.cuh"

namespace cr {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// deterministic single-block sum of per-thread values; result to out[q]
template <int NV>
__device__ void block_sum_store(double (&v)[NV], double* out) {
  __shared__ double scr[32 * NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) scr[wid * NV + q] = v[q];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = lane < nw ? scr[lane * NV + q] : 0.0;
      t = warp_sum(t);
      if (lane == 0) out[q] = t;
    }
  }
}

__global__ void zcoef_kernel(int j, const double* __restrict__ Z, int64_t ldz, int trans,
                             const double* __restrict__ h, double lam, double* __restrict__ g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * j) return;
  const int p = t / 3, s = t % 3;
  const double coef = s == 1 ? 2.0 * lam : lam;
  double acc = 0.0;
  for (int q = 0; q < j; ++q) {
    const double z = trans ? Z[q + (int64_t)p * ldz] : Z[p + (int64_t)q * ldz];
    acc = fma(z, h[3 * q + 2 - s], acc);
  }
  g[t] = coef * acc;
}

__global__ void mirror_col_kernel(int col, double* A, int64_t ld, int64_t stride) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= col) return;
  double* a = A + (int64_t)blockIdx.y * stride;
  a[col + (int64_t)p * ld] = a[p + (int64_t)col * ld];
}

__global__ void zero_border_kernel(int j, double* Z, int64_t ld) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > j) return;
  Z[j + (int64_t)q * ld] = 0.0;
  Z[q + (int64_t)j * ld] = 0.0;
}

__global__ void mask_residual_kernel(int64_t tot, int n, const double* __restrict__ OmY, const uint8_t* __restrict__ Om,
                                     int64_t ldo, double* E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int64_t i = t % n, a = t / n;
  E[t] = OmY[t] - (double)Om[i + a * ldo] * E[t];
}

__global__ void omega_times_kernel(int64_t tot, int n, const uint8_t* __restrict__ Om, int64_t ldo,
                                   const double* __restrict__ u, double* B) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int64_t i = t % n, a = t / n;
  B[t] = (double)Om[i + a * ldo] * u[i];
}

__global__ void mat_dot_kernel(int r, int c, const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                               int64_t ldb, double* out) {
  double v[1] = {0.0};
  const int64_t tot = (int64_t)r * c;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    const int64_t i = t % r, l = t / r;
    v[0] = fma(A[i + l * lda], B[i + l * ldb], v[0]);
  }
  block_sum_store<1>(v, out);
}

__global__ void mat_diff_kernel(int j, const double* __restrict__ Z, const double* __restrict__ Zp, int64_t ld,
                                double* out) {
  double v[2] = {0.0, 0.0};
  const int64_t tot = (int64_t)j * j;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    const int64_t i = t % j, l = t / j;
    const double z = Z[i + l * ld], d = z - Zp[i + l * ld];
    v[0] = fma(d, d, v[0]);
    v[1] = fma(z, z, v[1]);
  }
  block_sum_store<2>(v, out);
}

// out[0] = sum Om (P - Y)^2, out[1] = sum Om Y^2 over n x m (Om is 0/1)
__global__ void cv_err_kernel(int n, int m, const double* __restrict__ P, const double* __restrict__ Y,
                              const uint8_t* __restrict__ Om, double* out) {
  double v[2] = {0.0, 0.0};
  const int64_t tot = (int64_t)n * m;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    if (!Om[t]) continue;
    const double y = Y[t], d = P[t] - y;
    v[0] = fma(d, d, v[0]);
    v[1] = fma(y, y, v[1]);
  }
  block_sum_store<2>(v, out);
}

__global__ void mat_axpby_kernel(int r, int c, double alpha, const double* A, int64_t lda, double beta,
                                 const double* B, int64_t ldb, double* C, int64_t ldc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * c) return;
  const int64_t i = t % r, l = t / r;
  const double b = beta == 0.0 ? 0.0 : beta * B[i + l * ldb];
  C[i + l * ldc] = alpha * A[i + l * lda] + b;
}

__global__ void copy2d_kernel(int r, int c, const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                              int64_t ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * c) return;
  const int64_t i = t % r, l = t / r;
  dst[i + l * ldd] = src[i + l * lds];
}

__global__ void cg_zr_kernel(int j, double* Z, double* R, const double* __restrict__ P, const double* __restrict__ Q,
                             int64_t ld, const double* gs, int k) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)j * j) return;
  const double rho = gs[k & 1], pq = gs[2];
  const double alpha = (rho > 0.0 && pq > 0.0) ? rho / pq : 0.0;
  const int64_t o = (t % j) + (t / j) * ld;
  Z[o] = fma(alpha, P[o], Z[o]);
  R[o] = fma(-alpha, Q[o], R[o]);
}

__global__ void cg_p_kernel(int j, double* P, const double* __restrict__ R, int64_t ld, const double* gs, int k) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)j * j) return;
  const double rho_old = gs[k & 1], rho_new = gs[(k + 1) & 1];
  const double beta = rho_old > 0.0 ? rho_new / rho_old : 0.0;
  const int64_t o = (t % j) + (t / j) * ld;
  P[o] = fma(beta, P[o], R[o]);
}

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void zcoef(int j, const double* Z, int64_t ldz, int trans, const double* h, double lam, double* g, cudaStream_t st) {
  if (j <= 0) return;
  count_launch();
  zcoef_kernel<<<nblk(3 * j, 128), 128, 0, st>>>(j, Z, ldz, trans, h, lam, g);
}

void mirror_col(int col, double* A, int64_t ld, int batch, int64_t stride, cudaStream_t st) {
  if (col <= 0 || batch <= 0) return;
  count_launch();
  mirror_col_kernel<<<dim3(nblk(col, 128), batch), 128, 0, st>>>(col, A, ld, stride);
}

void zero_border(int j, double* Z, int64_t ld, cudaStream_t st) {
  count_launch();
  zero_border_kernel<<<nblk(j + 1, 128), 128, 0, st>>>(j, Z, ld);
}

void mask_residual(int n, int m, const double* OmY, const uint8_t* Om, int64_t ldo, double* E, cudaStream_t st) {
  const int64_t tot = (int64_t)n * m;
  if (tot == 0) return;
  count_launch();
  mask_residual_kernel<<<nblk(tot), 256, 0, st>>>(tot, n, OmY, Om, ldo, E);
}

void omega_times(int n, int m, const uint8_t* Om, int64_t ldo, const double* u, double* B, cudaStream_t st) {
  const int64_t tot = (int64_t)n * m;
  if (tot == 0) return;
  count_launch();
  omega_times_kernel<<<nblk(tot), 256, 0, st>>>(tot, n, Om, ldo, u, B);
}

void mat_dot(int r, int c, const double* A, int64_t lda, const double* B, int64_t ldb, double* out, cudaStream_t st) {
  count_launch();
  mat_dot_kernel<<<1, 1024, 0, st>>>(r, c, A, lda, B, ldb, out);
}

void cv_err(int n, int m, const double* P, const double* Y, const uint8_t* Om, double* out, cudaStream_t st) {
  count_launch();
  cv_err_kernel<<<1, 1024, 0, st>>>(n, m, P, Y, Om, out);
}

void mat_diff_norms(int j, const double* Z, const double* Zp, int64_t ld, double* out, cudaStream_t st) {
  count_launch();
  mat_diff_kernel<<<1, 1024, 0, st>>>(j, Z, Zp, ld, out);
}

void mat_axpby(int r, int c, double alpha, const double* A, int64_t lda, double beta, const double* B, int64_t ldb,
               double* C, int64_t ldc, cudaStream_t st) {
  const int64_t tot = (int64_t)r * c;
  if (tot == 0) return;
  count_launch();
  mat_axpby_kernel<<<nblk(tot), 256, 0, st>>>(r, c, alpha, A, lda, beta, B, ldb, C, ldc);
}

void copy2d(int r, int c, const double* src, int64_t lds, double* dst, int64_t ldd, cudaStream_t st) {
  const int64_t tot = (int64_t)r * c;
  if (tot == 0) return;
  count_launch();
  copy2d_kernel<<<nblk(tot), 256, 0, st>>>(r, c, src, lds, dst, ldd);
}

void cg_update_zr(int j, double* Z, double* R, const double* P, const double* Q, int64_t ld, const double* gs, int k,
                  cudaStream_t st) {
  count_launch();
  cg_zr_kernel<<<nblk((int64_t)j * j), 256, 0, st>>>(j, Z, R, P, Q, ld, gs, k);
}

void cg_update_p(int j, double* P, const double* R, int64_t ld, const double* gs, int k, cudaStream_t st) {
  count_launch();
  cg_p_kernel<<<nblk((int64_t)j * j), 256, 0, st>>>(j, P, R, ld, gs, k);
}

}  // namespace cr

namespace cr {
namespace {

// Diagonal of the projected operator of Eq. (Proj_Sylv) acting on Z(p, q):
//   lam (B2_qq + 2 A1_pp B1_qq + A2_pp) + sum_a G_a,pp H_qa^2
__global__ void galerkin_diag_kernel(int j, int m, const double* __restrict__ A1, const double* __restrict__ A2,
                                     const double* __restrict__ B1, const double* __restrict__ B2,
                                     const double* __restrict__ G, const double* __restrict__ H, int64_t ld,
                                     double lam, double* __restrict__ Dg) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)j * j) return;
  const int pp = (int)(t % j), q = (int)(t / j);
  double v = lam * (B2[q + q * ld] + 2.0 * A1[pp + pp * ld] * B1[q + q * ld] + A2[pp + pp * ld]);
  for (int a = 0; a < m; ++a) {
    const double h = H[q + (int64_t)a * ld];
    v = fma(G[(int64_t)a * ld * ld + pp + pp * ld] * h, h, v);
  }
  Dg[pp + q * ld] = v > 0.0 ? v : 1.0;
}

// Zp = R ./ Dg; out[0] = <R, Zp>, out[1] = <R, R> (one block, fixed order)
__global__ void precond_dots_kernel(int j, const double* __restrict__ R, const double* __restrict__ Dg, int64_t ld,
                                    double* __restrict__ Zp, double* out0, double* out1) {
  __shared__ double scr[64];
  double a = 0.0, b = 0.0;
  const int64_t tot = (int64_t)j * j;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    const int64_t o = (t % j) + (t / j) * ld;
    const double r = R[o];
    const double z = r / Dg[o];
    Zp[o] = z;
    a = fma(r, z, a);
    b = fma(r, r, b);
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, s);
    b += __shfl_down_sync(0xffffffffu, b, s);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    scr[wid] = a;
    scr[32 + wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < nw ? scr[lane] : 0.0;
    b = lane < nw ? scr[32 + lane] : 0.0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, s);
      b += __shfl_down_sync(0xffffffffu, b, s);
    }
    if (lane == 0) {
      *out0 = a;
      *out1 = b;
    }
  }
}

}  // namespace

void galerkin_diag(int j, int m, const double* A1, const double* A2, const double* B1, const double* B2,
                   const double* G, const double* H, int64_t ld, double lam, double* Dg, cudaStream_t st) {
  const int64_t tot = (int64_t)j * j;
  if (tot == 0) return;
  count_launch();
  galerkin_diag_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(j, m, A1, A2, B1, B2, G, H, ld, lam, Dg);
}

void precond_dots(int j, const double* R, const double* Dg, int64_t ld, double* Zp, double* out0, double* out1,
                  cudaStream_t st) {
  count_launch();
  precond_dots_kernel<<<1, 1024, 0, st>>>(j, R, Dg, ld, Zp, out0, out1);
}

}  // namespace cr

namespace cr {
namespace {
__global__ void to_f32_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
__global__ void add_f32_kernel(int r, int c, const float* __restrict__ x, int64_t ldx, double* __restrict__ y,
                               int64_t ldy) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * c) return;
  const int64_t i = t % r, l = t / r;
  y[i + l * ldy] += (double)x[i + l * ldx];
}
}  // namespace

void to_f32(int64_t n, const double* x, float* y, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y);
}

void add_f32(int r, int c, const float* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  const int64_t tot = (int64_t)r * c;
  if (tot <= 0) return;
  count_launch();
  add_f32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r, c, x, ldx, y, ldy);
}
}  // namespace cr
