// Arrowhead eigen-decomposition on the device: the step that keeps the
// eigenbases of U^T L_y U and V^T L_x V up to date as the Galerkin projection
// (Eq. Proj_Sylv) grows by one border per greedy step.  For
//
//   M = [ diag(d)  z ]      d ascending (the current eigenvalues), z = Q^T a,
//       [ z^T  alpha ]      alpha the new diagonal entry,
//
// M = W diag(mu) W^T, and the bordered matrix's eigenbasis is blockdiag(Q, 1) W.
// The method is that of the secular equation of a rank-one bordering:
//   - entries with negligible z_i, and one of each pair of nearly equal poles
//     (after a plane rotation that moves its coupling onto the other), are
//     deflated and keep (d_i, e_i);
//   - the k remaining poles give k + 1 roots of
//       f(mu) = alpha - mu - sum_t z_t^2 / (d_t - mu),
//     one between consecutive poles and one beyond each end, where f decreases;
//     each is found by Newton steps kept inside its bracket by bisection;
//   - the eigenvectors come from the coupling recomputed from the computed roots
//     (the Loewner construction of Gu and Eisenstat), which keeps them
//     numerically orthogonal however close the roots are.
// Both sides (blockIdx.y = 0: A1, 1: B1) run in the same launches, with no host
// round trip.
#include "cr_common.cuh"

namespace cr {
namespace {

constexpr double kEps = 2.2204460492503131e-16;

// per-side work layout (doubles): dc, zz, dl, zl, zh, rc, rs (n each), root (n + 1);
// then ints: live, dfl, ra, rb (n each), meta[4] = {k, nrot, ndefl, identity}
struct ArrowWork {
  double *dc, *zz, *dl, *zl, *zh, *rc, *rs, *root, *scal;
  int *live, *dfl, *ra, *rb, *meta;
};

__device__ ArrowWork work_of(double* base, int nmax) {
  const int64_t n1 = nmax + 1;
  ArrowWork w;
  double* q = base;
  w.dc = q; q += n1;
  w.zz = q; q += n1;
  w.dl = q; q += n1;
  w.zl = q; q += n1;
  w.zh = q; q += n1;
  w.rc = q; q += n1;
  w.rs = q; q += n1;
  w.root = q; q += n1;
  w.scal = q; q += 4;
  int* iq = reinterpret_cast<int*>(q);
  w.live = iq; iq += n1;
  w.dfl = iq; iq += n1;
  w.ra = iq; iq += n1;
  w.rb = iq; iq += n1;
  w.meta = iq;
  return w;
}

struct ArrowArgs {
  int n, nmax;
  const double* d[2];      // eigenvalues (n)
  const double* z[2];      // couplings (n)
  const double* alpha[2];  // device scalar
  double* mu[2];           // n + 1 (may alias d: read before written)
  double* W[2];            // (n + 1)^2, column-major, ld n + 1
  double* work;            // 2 sides x arrow_work_doubles(nmax)
  int64_t side_stride;
};

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    red[32] = t;
  }
  __syncthreads();
  const double t = red[32];
  __syncthreads();
  return t;
}

// Deflation and compaction (one CTA per side; the pole pass is sequential).
__global__ void arrow_prep_kernel(ArrowArgs a) {
  const int s = blockIdx.y, n = a.n;
  ArrowWork w = work_of(a.work + s * a.side_stride, a.nmax);
  extern __shared__ double sm[];
  double* d = sm;                            // n
  double* zz = d + n;                        // n
  char* defl = reinterpret_cast<char*>(zz + n);
  __shared__ double red[33];
  const double alpha = *a.alpha[s];
  double mx = fabs(alpha);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = a.d[s][i], zi = a.z[s][i];
    d[i] = di;
    zz[i] = zi;
    w.dc[i] = di;
    mx = fmax(mx, fmax(fabs(di), fabs(zi)));
  }
  const double scale = block_max(mx, red);
  const double tol = 8.0 * kEps * scale;
  for (int i = threadIdx.x; i < n; i += blockDim.x) defl[i] = fabs(zz[i]) <= tol ? 1 : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int nrot = 0, last = -1;
    for (int i = 0; i < n; ++i) {
      if (defl[i]) continue;
      if (last >= 0 && fabs(d[i] - d[last]) <= tol) {
        const double r = hypot(zz[last], zz[i]);
        w.ra[nrot] = last;
        w.rb[nrot] = i;
        w.rc[nrot] = zz[i] / r;
        w.rs[nrot] = zz[last] / r;
        ++nrot;
        zz[last] = 0.0;
        zz[i] = r;
        defl[last] = 1;
      }
      last = i;
    }
    int k = 0, nd = 0;
    double zn2 = 0.0;
    for (int i = 0; i < n; ++i) {
      if (defl[i]) {
        w.dfl[nd++] = i;
      } else {
        w.live[k] = i;
        w.dl[k] = d[i];
        w.zl[k] = zz[i];
        zn2 += zz[i] * zz[i];
        ++k;
      }
    }
    w.meta[0] = k;
    w.meta[1] = nrot;
    w.meta[2] = nd;
    w.meta[3] = scale == 0.0 ? 1 : 0;
    w.scal[0] = alpha;
    w.scal[1] = sqrt(zn2);
    w.scal[2] = scale;
  }
}

// Secular roots, one warp per root r = 0..k.
__global__ void arrow_roots_kernel(ArrowArgs a) {
  const int s = blockIdx.y;
  ArrowWork w = work_of(a.work + s * a.side_stride, a.nmax);
  const int k = w.meta[0];
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r > k || w.meta[3]) return;
  const double alpha = w.scal[0], zn = w.scal[1], scale = w.scal[2];
  if (k == 0) {
    if (lane == 0) w.root[0] = alpha;
    return;
  }
  double lo, hi;
  if (r == 0) {
    lo = fmin(w.dl[0], alpha) - zn - scale * kEps;
    hi = w.dl[0];
  } else if (r == k) {
    lo = w.dl[k - 1];
    hi = fmax(w.dl[k - 1], alpha) + zn + scale * kEps;
  } else {
    lo = w.dl[r - 1];
    hi = w.dl[r];
  }
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double fv = 0.0, fd = 0.0;
    for (int t = lane; t < k; t += 32) {
      const double q = 1.0 / (w.dl[t] - x), y = w.zl[t] * q;
      fv -= w.zl[t] * y;
      fd -= y * y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      fv += __shfl_xor_sync(0xffffffffu, fv, o);
      fd += __shfl_xor_sync(0xffffffffu, fd, o);
    }
    fv += alpha - x;
    fd -= 1.0;
    if (fv > 0.0)
      lo = x;
    else
      hi = x;
    if (fv == 0.0) break;
    double xn = x - fv / fd;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (xn == x || !(xn > lo && xn < hi)) break;
    if (fabs(xn - x) <= 4.0 * kEps * fmax(fabs(xn), fabs(x))) {
      x = xn;
      break;
    }
    x = xn;
  }
  if (lane == 0) w.root[r] = x;
}

// Loewner couplings: zh_t^2 = -prod_r (root_r - d_t) / prod_{s != t} (d_s - d_t).
__global__ void arrow_zhat_kernel(ArrowArgs a) {
  const int s = blockIdx.y;
  ArrowWork w = work_of(a.work + s * a.side_stride, a.nmax);
  const int k = w.meta[0];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k || w.meta[3]) return;
  const double dt = w.dl[t];
  double p = w.root[k] - dt;
  for (int r = 0; r < k; ++r) {
    p *= (w.root[r] - dt);
    if (r != t) p /= (w.dl[r] - dt);
  }
  w.zh[t] = copysign(sqrt(fabs(p)), w.zl[t]);
}

// Eigenvectors, one warp per eigenpair: deflated pairs (d_i, e_i) and the k + 1
// secular pairs, written to their place in ascending order (deflated first among
// equal values); then the recorded rotations are undone on that column.
__global__ void arrow_vectors_kernel(ArrowArgs a) {
  const int s = blockIdx.y, n = a.n, N = n + 1;
  ArrowWork w = work_of(a.work + s * a.side_stride, a.nmax);
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= N) return;
  double* W = a.W[s];
  if (w.meta[3]) {  // M == 0: identity
    for (int q = lane; q < N; q += 32) W[q + (int64_t)c * N] = q == c ? 1.0 : 0.0;
    if (lane == 0) a.mu[s][c] = 0.0;
    return;
  }
  const int k = w.meta[0], nrot = w.meta[1], nd = w.meta[2];
  double val;
  int pos;
  if (c < nd) {  // deflated: e_i with value d_i
    const int i = w.dfl[c];
    val = w.dc[i];
    int lo = 0, hi = k + 1;  // roots strictly below val
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (w.root[mid] < val) lo = mid + 1; else hi = mid;
    }
    pos = c + lo;
  } else {
    const int r = c - nd;
    val = w.root[r];
    int lo = 0, hi = nd;  // deflated values at or below val
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (w.dc[w.dfl[mid]] <= val) lo = mid + 1; else hi = mid;
    }
    pos = r + lo;
  }
  double* col = W + (int64_t)pos * N;
  for (int q = lane; q < N; q += 32) col[q] = 0.0;
  __syncwarp();
  if (c < nd) {
    if (lane == 0) col[w.dfl[c]] = 1.0;
  } else {
    const int r = c - nd;
    const double x = w.root[r];
    double nrm = 0.0;
    for (int t = lane; t < k; t += 32) {
      const double y = w.zh[t] / (w.dl[t] - x);
      col[w.live[t]] = y;
      nrm += y * y;
    }
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    const double inv = 1.0 / sqrt(nrm + 1.0);  // last component -1
    __syncwarp();
    for (int t = lane; t < k; t += 32) col[w.live[t]] *= inv;
    if (lane == 0) col[n] = -inv;
  }
  __syncwarp();
  if (lane == 0) {
    for (int q = nrot - 1; q >= 0; --q) {
      const int ia = w.ra[q], ib = w.rb[q];
      const double cc = w.rc[q], ss = w.rs[q];
      const double va = col[ia], vb = col[ib];
      col[ia] = cc * va + ss * vb;
      col[ib] = -ss * va + cc * vb;
    }
    a.mu[s][pos] = val;
  }
}

}  // namespace

size_t arrow_work_doubles(int nmax) {
  const size_t n1 = (size_t)nmax + 1;
  return 8 * n1 + 4 + (4 * n1 + 4 + 1) / 2 + 1;
}

cudaError_t arrow_update(int n, int nmax, const double* const d[2], const double* const z[2],
                         const double* const alpha[2], double* const mu[2], double* const W[2], double* work,
                         cudaStream_t st) {
  if (n < 0 || n > nmax) return cudaErrorInvalidValue;
  ArrowArgs a{};
  a.n = n;
  a.nmax = nmax;
  for (int s = 0; s < 2; ++s) {
    a.d[s] = d[s];
    a.z[s] = z[s];
    a.alpha[s] = alpha[s];
    a.mu[s] = mu[s];
    a.W[s] = W[s];
  }
  a.work = work;
  a.side_stride = (int64_t)arrow_work_doubles(nmax);
  const size_t smem = (size_t)n * (2 * sizeof(double) + 1) + 16;
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(arrow_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launch();
  arrow_prep_kernel<<<dim3(1, 2), 256, smem, st>>>(a);
  const int wpb = 8;  // warps per block
  count_launch();
  arrow_roots_kernel<<<dim3((n + 1 + wpb - 1) / wpb, 2), 32 * wpb, 0, st>>>(a);
  if (n > 0) {
    count_launch();
    arrow_zhat_kernel<<<dim3((n + 127) / 128, 2), 128, 0, st>>>(a);
  }
  count_launch();
  arrow_vectors_kernel<<<dim3((n + 1 + wpb - 1) / wpb, 2), 32 * wpb, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace cr

extern "C" cr_status cr_arrow_check(int32_t n, const double* d, const double* z, double alpha, double* mu,
                                    double* W) {
  if (n < 0 || n > 4096 || (n > 0 && (!d || !z)) || !mu || !W) return CR_EINVAL;
  const int n1 = n + 1;
  const size_t wk = cr::arrow_work_doubles(n);
  const size_t total = 2 * (size_t)n + 1 + 2 * (size_t)n1 + 2 * (size_t)n1 * n1 + 2 * wk;
  double* blk = nullptr;
  cudaStream_t st = nullptr;
  if (cudaMalloc(&blk, sizeof(double) * total) != cudaSuccess) {
    cudaGetLastError();
    return CR_ENOMEM;
  }
  cr_status rc = CR_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(blk);
    return CR_ECUDA;
  }
  double* dd = blk;
  double* dz = dd + n;
  double* dal = dz + n;
  double* dmu = dal + 1;  // two sides
  double* dW = dmu + 2 * (size_t)n1;
  double* work = dW + 2 * (size_t)n1 * n1;
  cudaMemsetAsync(blk, 0, sizeof(double) * total, st);
  if (n > 0) {
    cudaMemcpyAsync(dd, d, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dz, z, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  }
  cudaMemcpyAsync(dal, &alpha, sizeof(double), cudaMemcpyHostToDevice, st);
  const double* ds[2] = {dd, dd};
  const double* zs[2] = {dz, dz};
  const double* as[2] = {dal, dal};
  double* ms[2] = {dmu, dmu + n1};
  double* Ws[2] = {dW, dW + (size_t)n1 * n1};
  if (cr::arrow_update(n, n, ds, zs, as, ms, Ws, work, st) != cudaSuccess) rc = CR_ECUDA;
  cudaMemcpyAsync(mu, dmu, sizeof(double) * n1, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(W, dW, sizeof(double) * n1 * n1, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = CR_ECUDA;
  cudaStreamDestroy(st);
  cudaFree(blk);
  return rc;
}
