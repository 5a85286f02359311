// Kernels of the flexible CG used with the learned preconditioner (Sec. 2.3
// sub-problems, Eqs. ALS_linsys / ALS_linsys_v):
//   operator  lam [(L + cI)^2 + (d - c^2) I] + data,  data = diag(omega) (u side)
//             or X diag(s) X^T (v side), with c, d read on the device;
//   preconditioner  z = D^-1 r + s net(D^-1 r / s, mask),  s = |D^-1 r|,
//   where the network runs on the voxel box (cr_net.cu).
// Scalars stay on the device; the host checks convergence every few steps.
#include "cr_common.cuh"

namespace cr {
namespace {

__device__ __forceinline__ double lap_row(const DevLap& L, int i, const double* v, double shift) {
  double acc = (L.diag[i] + shift) * v[i];
  for (int k = 0; k < L.K; ++k) {
    const int q = L.nbr[(size_t)k * L.n + i];
    if (q < 0) continue;
    acc += (L.offw ? L.offw[(size_t)k * L.n + i] : -1.0) * v[q];
  }
  return acc;
}

// Jacobi diagonal of the operator; u side also stores omega = sum_a Om_ia xi_a^2
__global__ void jacobi_diag_kernel(DevLap L, double lam, const double* coef, int side, int m, const uint8_t* Om,
                                   int64_t ldo, const double* xi, const int* xr_ptr, const int* xr_col,
                                   const double* xr_val, const double* s, double* omt, double* dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  const double c = coef[0], d = coef[1];
  double dd = lam * (L.l2diag[i] + 2.0 * c * L.diag[i] + d);
  if (side == 0) {
    double o = 0.0;
    for (int a = 0; a < m; ++a) o += (double)Om[i + (int64_t)a * ldo] * xi[a] * xi[a];
    omt[i] = o;
    dd += o;
  } else {
    for (int q = xr_ptr[i]; q < xr_ptr[i + 1]; ++q) dd += xr_val[q] * xr_val[q] * s[xr_col[q]];
  }
  dinv[i] = dd > 0.0 ? 1.0 / dd : 1.0;
}

__global__ void shift_lap_kernel(DevLap L, const double* coef, const double* p, double* t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  t[i] = lap_row(L, i, p, coef[0]);
}

// out = lam ((L + cI) t + (d - c^2) p) + data(p); y = X^T p for the v side
__global__ void ahat_out_kernel(DevLap L, double lam, const double* coef, const double* t, const double* p, int side,
                                const double* omt, const int* xr_ptr, const int* xr_col, const double* xr_val,
                                const double* s, const double* y, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  const double c = coef[0], e = coef[1] - c * c;
  double w = lam * (lap_row(L, i, t, c) + e * p[i]);
  if (side == 0) {
    w += omt[i] * p[i];
  } else {
    for (int q = xr_ptr[i]; q < xr_ptr[i + 1]; ++q) w += xr_val[q] * s[xr_col[q]] * y[xr_col[q]];
  }
  out[i] = w;
}

// network input: in[0][box_i] = dinv_i r_i / s, in[1][box_i] = 1 (float32)
__global__ void net_input_kernel(int n, const int* box, const double* dinv, const double* r, const double* s2,
                                 float* in, int64_t V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = sqrt(*s2);
  in[box[i]] = (float)(s > 0.0 ? dinv[i] * r[i] / s : 0.0);
  in[V + box[i]] = 1.f;
}

__global__ void dinv_r_kernel(int n, const double* dinv, const double* r, double* z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = dinv[i] * r[i];
}

// z = dinv r + s net_out[box]
__global__ void net_output_kernel(int n, const int* box, const double* dinv, const double* r, const double* s2,
                                  const float* out, double* z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = dinv[i] * r[i] + sqrt(*s2) * (double)out[box[i]];
}

// sc: [0] rho = <r, z>, [1] pq, [2] |r|^2, [3] <z_new, r_new - r_old>, [4] s^2
__global__ void fcg_xr_kernel(int n, double* x, double* r, double* rold, const double* p, const double* q,
                              const double* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double alpha = sc[1] > 0.0 ? sc[0] / sc[1] : 0.0;
  x[i] += alpha * p[i];
  rold[i] = r[i];
  r[i] -= alpha * q[i];
}

__global__ void fcg_diff_kernel(int n, const double* r, const double* rold, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = r[i] - rold[i];
}

// p = z + beta p, beta = <z_new, r_new - r_old> / rho_old (Polak-Ribiere); then rho = <r, z> is recomputed
__global__ void fcg_p_kernel(int n, double* p, const double* z, const double* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double beta = sc[0] > 0.0 ? sc[3] / sc[0] : 0.0;
  p[i] = z[i] + beta * p[i];
}

inline unsigned nb256(int n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void fcg_jacobi_diag(const DevLap& L, double lam, const double* coef, int side, int m, const uint8_t* Om, int64_t ldo,
                     const double* xi, const DevXLocal& X, const double* s, double* omt, double* dinv,
                     cudaStream_t st) {
  count_launch();
  jacobi_diag_kernel<<<nb256(L.n), 256, 0, st>>>(L, lam, coef, side, m, Om, ldo, xi, X.xr_ptr, X.xr_col, X.xr_val, s,
                                                 omt, dinv);
}

void fcg_apply(const DevLap& L, double lam, const double* coef, int side, const double* omt, const DevXLocal& X,
               const int* xc_ptr, const int* xc_row, const double* xc_val, int m, const double* s, double* y,
               const double* p, double* t, double* out, cudaStream_t st) {
  count_launch();
  shift_lap_kernel<<<nb256(L.n), 256, 0, st>>>(L, coef, p, t);
  if (side == 1) spmv_xt(m, xc_ptr, xc_row, xc_val, p, y, 1, st);
  count_launch();
  ahat_out_kernel<<<nb256(L.n), 256, 0, st>>>(L, lam, coef, t, p, side, omt, X.xr_ptr, X.xr_col, X.xr_val, s, y, out);
}

void fcg_precond(int n, const int* box, const double* dinv, const double* r, double* s2, float* in, int64_t V,
                 cr_net* net, float* out, double* z, cudaStream_t st) {
  if (!net) {
    count_launch();
    dinv_r_kernel<<<nb256(n), 256, 0, st>>>(n, dinv, r, z);
    return;
  }
  count_launch();
  dinv_r_kernel<<<nb256(n), 256, 0, st>>>(n, dinv, r, z);
  dot(n, z, z, s2, st);
  cudaMemsetAsync(in, 0, sizeof(float) * 2 * V, st);
  count_launch();
  net_input_kernel<<<nb256(n), 256, 0, st>>>(n, box, dinv, r, s2, in, V);
  net_apply(net, in, out, st);
  count_launch();
  net_output_kernel<<<nb256(n), 256, 0, st>>>(n, box, dinv, r, s2, out, z);
}

void fcg_update_xr(int n, double* x, double* r, double* rold, const double* p, const double* q, const double* sc,
                   cudaStream_t st) {
  count_launch();
  fcg_xr_kernel<<<nb256(n), 256, 0, st>>>(n, x, r, rold, p, q, sc);
}

void fcg_diff(int n, const double* r, const double* rold, double* d, cudaStream_t st) {
  count_launch();
  fcg_diff_kernel<<<nb256(n), 256, 0, st>>>(n, r, rold, d);
}

void fcg_update_p(int n, double* p, const double* z, const double* sc, cudaStream_t st) {
  count_launch();
  fcg_p_kernel<<<nb256(n), 256, 0, st>>>(n, p, z, sc);
}

}  // namespace cr
