// Persistent Galerkin CG (Eq. Proj_Sylv) in one cooperative launch.
//
// The projected operator
//   K(X) = lam (X B2 + 2 A1 X B1 + A2 X) + sum_a G_a X h_a h_a^T
// is small (j <= a few hundred) but is applied hundreds of times per
// projection; issued as separate GEMM launches each CG iteration costs a dozen
// launches.  Here one grid of one CTA per SM runs the whole Jacobi-preconditioned
// matrix CG.  Each iteration has five phases separated by a grid barrier:
//   A  T2 = X B2, T1 = X B1, TH = X H              (8x8 output tiles)
//   B  Gw(:, a) = G_a TH(:, a)                       (64-row tiles per a)
//   C  Q = lam T2 + 2 lam A1 T1 + lam A2 X + Gw H^T  (8x8 tiles) and <X, Q>
//   D  alpha; Z += alpha X; R -= alpha Q; z = R ./ diag(K); <R, z>, <R, R>
//   E  beta; X_next = z + beta X
// Tiles use all CTAs; each output is summed in a fixed order (k split in four
// fixed ranges added in order), and every CTA adds the per-CTA partial sums of
// the inner products in block order, so all CTAs take the same decisions and
// the result is bitwise reproducible.  Data produced by other CTAs in the same
// launch is read with ld.global.cg (L2), never from a possibly stale L1 line.
// The grid barrier spins with a bound; on timeout it raises an error word that
// makes every CTA leave, and the host reports CR_ETIMEOUT.
#include "cr_common.cuh"

namespace cr {

namespace {

constexpr int kGThreads = 256;
constexpr int TS = 8;

struct GalArgs {
  int j, m, nb;
  int64_t ld;
  double lam;
  const double *A1, *A2, *B1, *B2, *G, *H, *F, *Dg;
  double *Z, *R, *Pa, *Pb, *Q, *T2, *T1, *TH, *Gw, *zb;
  double* part;        // [nb * 4]
  unsigned* bar;       // [0] arrivals, [1] generation
  int* err;            // timeout flag
  double tol2;         // stop when |R|^2 <= tol2
  int maxit;
  double* out;         // [0] iterations, [1] |R|^2, [2] status (0 ok, 1 cap, 2 breakdown, 3 barrier timeout)
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Grid-wide barrier with a bounded spin.  Returns false if the error word is set.
__device__ __forceinline__ bool grid_barrier(const GalArgs& a) {
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
        if (++spins > (1ll << 24)) {  // ~ seconds: something is wrong; let everyone leave
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the CTA (fixed order) and store them at part[blockIdx * 4 + q].
template <int NV>
__device__ void cta_partial(double (&v)[NV], const GalArgs& a) {
  __shared__ double scr[32 * 4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) scr[wid * 4 + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += scr[w * 4 + q];
      a.part[blockIdx.x * 4 + q] = t;
    }
  }
}

// After a barrier: totals of the per-CTA partials, same order in every CTA.
template <int NV>
__device__ void grid_total(const GalArgs& a, double (&out)[NV]) {
  __shared__ double tot[4];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      for (int b = lane; b < a.nb; b += 32) t += ldcg(a.part + b * 4 + q);
      t = warp_sum(t);
      if (lane == 0) tot[q] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = tot[q];
  __syncthreads();
}

// One 8x8 output tile of sum_k A(i, k) B(k, l); 256 threads = 64 outputs x 4
// k-groups.  Returns this thread's partial; combine with tile_reduce.
template <class GA, class GB>
__device__ __forceinline__ double tile_term(int i0, int l0, int M, int N, int K, GA ga, GB gb, double acc) {
  __shared__ double As[32][TS + 1];
  __shared__ double Bs[32][TS + 1];
  const int tid = threadIdx.x;
  const int o = tid & 63, g = tid >> 6;
  const int oi = o & 7, ol = o >> 3;
  for (int k0 = 0; k0 < K; k0 += 32) {
    {
      const int ii = tid & 7, kk = tid >> 3;
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < M && k < K) ? ga(i, k) : 0.0;
    }
    {
      const int kk = tid & 31, ll = tid >> 5;
      const int l = l0 + ll, k = k0 + kk;
      Bs[kk][ll] = (l < N && k < K) ? gb(k, l) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) acc = fma(As[g * 8 + q][oi], Bs[g * 8 + q][ol], acc);
    __syncthreads();
  }
  return acc;
}

// Add the 4 k-group partials in order; threads 0..63 return the output of
// (i0 + (t & 7), l0 + (t >> 3)), others return 0 with valid = false.
__device__ __forceinline__ double tile_reduce(double acc, bool& valid) {
  __shared__ double red[4][64];
  const int tid = threadIdx.x;
  red[tid >> 6][tid & 63] = acc;
  __syncthreads();
  double v = 0.0;
  valid = tid < 64;
  if (valid) v = ((red[0][tid] + red[1][tid]) + red[2][tid]) + red[3][tid];
  __syncthreads();
  return v;
}

// K(X) -> Q for X = Xin (phases A, B, C); returns <X, Q> partial of this CTA in pq.
__device__ bool apply_K(const GalArgs& a, const double* X, double& pq) {
  const int j = a.j, m = a.m;
  const int64_t ld = a.ld;
  const int nt = (j + TS - 1) / TS, ntm = (m + TS - 1) / TS;
  // A
  const int itemsA = 2 * nt * nt + nt * ntm;
  for (int it = blockIdx.x; it < itemsA; it += a.nb) {
    int which, ti, tl;
    if (it < nt * nt) {
      which = 0; ti = it % nt; tl = it / nt;
    } else if (it < 2 * nt * nt) {
      which = 1; ti = (it - nt * nt) % nt; tl = (it - nt * nt) / nt;
    } else {
      which = 2; ti = (it - 2 * nt * nt) % nt; tl = (it - 2 * nt * nt) / nt;
    }
    const int N = which == 2 ? m : j;
    const double* Bm = which == 0 ? a.B2 : which == 1 ? a.B1 : a.H;
    double* out = which == 0 ? a.T2 : which == 1 ? a.T1 : a.TH;
    double acc = tile_term(ti * TS, tl * TS, j, N, j, [&](int i, int k) { return ldcg(X + i + k * ld); },
                           [&](int k, int l) { return Bm[k + l * ld]; }, 0.0);
    bool v;
    const double r = tile_reduce(acc, v);
    if (v) {
      const int i = ti * TS + (threadIdx.x & 7), l = tl * TS + (threadIdx.x >> 3);
      if (i < j && l < N) out[i + l * ld] = r;
    }
  }
  if (!grid_barrier(a)) return false;
  // B
  const int nr = (j + 63) / 64;
  for (int it = blockIdx.x; it < m * nr; it += a.nb) {
    const int al = it / nr, rt = it % nr;
    const int i = rt * 64 + (threadIdx.x & 63), g = threadIdx.x >> 6;
    const double* Ga = a.G + (int64_t)al * ld * ld;
    double acc = 0.0;
    if (i < j) {
      const int q0 = g * ((j + 3) / 4), q1 = min(j, q0 + (j + 3) / 4);
      for (int q = q0; q < q1; ++q) acc = fma(Ga[i + q * ld], ldcg(a.TH + q + al * ld), acc);
    }
    __shared__ double rb[4][64];
    rb[g][threadIdx.x & 63] = acc;
    __syncthreads();
    if (threadIdx.x < 64 && i < j)
      a.Gw[i + (int64_t)al * ld] = ((rb[0][threadIdx.x] + rb[1][threadIdx.x]) + rb[2][threadIdx.x]) + rb[3][threadIdx.x];
    __syncthreads();
  }
  if (!grid_barrier(a)) return false;
  // C
  double dotpq = 0.0;
  const double lam = a.lam;
  for (int it = blockIdx.x; it < nt * nt; it += a.nb) {
    const int ti = it % nt, tl = it / nt;
    const int i0 = ti * TS, l0 = tl * TS;
    double acc = 0.0;
    acc = tile_term(i0, l0, j, j, j, [&](int i, int k) { return 2.0 * lam * a.A1[i + k * ld]; },
                    [&](int k, int l) { return ldcg(a.T1 + k + l * ld); }, acc);
    acc = tile_term(i0, l0, j, j, j, [&](int i, int k) { return lam * a.A2[i + k * ld]; },
                    [&](int k, int l) { return ldcg(X + k + l * ld); }, acc);
    acc = tile_term(i0, l0, j, j, m, [&](int i, int k) { return ldcg(a.Gw + i + k * ld); },
                    [&](int k, int l) { return a.H[l + k * ld]; }, acc);
    bool v;
    const double r = tile_reduce(acc, v);
    if (v) {
      const int i = i0 + (threadIdx.x & 7), l = l0 + (threadIdx.x >> 3);
      if (i < j && l < j) {
        const int64_t o = i + l * ld;
        const double q = fma(lam, ldcg(a.T2 + o), r);
        a.Q[o] = q;
        dotpq = fma(ldcg(X + o), q, dotpq);
      }
    }
  }
  pq = dotpq;
  return true;
}

__global__ void __launch_bounds__(kGThreads, 1) galerkin_cg_kernel(const GalArgs a) {
  const int j = a.j;
  const int64_t ld = a.ld;
  const int64_t tot = (int64_t)j * j;
  const int64_t chunk = (tot + a.nb - 1) / a.nb;
  const int64_t e0 = min(tot, (int64_t)blockIdx.x * chunk), e1 = min(tot, e0 + chunk);
  int status = 0, k = 0;
  double rho = 0.0, rr = 0.0;
  // initial residual R = F - K(Z), z = R ./ D, P = z
  double pq;
  if (!apply_K(a, a.Z, pq)) goto timeout;
  if (!grid_barrier(a)) goto timeout;
  {
    double v[2] = {0.0, 0.0};
    for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
      const int64_t o = (t % j) + (t / j) * ld;
      const double r = a.F[o] - ldcg(a.Q + o);
      const double z = r / a.Dg[o];
      a.R[o] = r;
      a.Pa[o] = z;
      v[0] = fma(r, z, v[0]);
      v[1] = fma(r, r, v[1]);
    }
    cta_partial<2>(v, a);
  }
  if (!grid_barrier(a)) goto timeout;
  {
    double t2[2];
    grid_total<2>(a, t2);
    rho = t2[0];
    rr = t2[1];
  }
  {
    double* X = a.Pa;
    double* Xn = a.Pb;
    while (rr > a.tol2) {
      if (k >= a.maxit) {
        status = 1;
        break;
      }
      if (!apply_K(a, X, pq)) goto timeout;
      {
        double v[1] = {pq};
        cta_partial<1>(v, a);
      }
      if (!grid_barrier(a)) goto timeout;
      double pqt[1];
      grid_total<1>(a, pqt);
      if (!(pqt[0] > 0.0) || !isfinite(pqt[0])) {
        status = 2;
        break;
      }
      const double alpha = rho / pqt[0];
      {
        double v[2] = {0.0, 0.0};
        for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
          const int64_t o = (t % j) + (t / j) * ld;
          a.Z[o] = fma(alpha, ldcg(X + o), a.Z[o]);
          const double r = fma(-alpha, ldcg(a.Q + o), a.R[o]);
          a.R[o] = r;
          const double z = r / a.Dg[o];
          a.zb[o] = z;
          v[0] = fma(r, z, v[0]);
          v[1] = fma(r, r, v[1]);
        }
        cta_partial<2>(v, a);
      }
      if (!grid_barrier(a)) goto timeout;
      double t2[2];
      grid_total<2>(a, t2);
      const double beta = rho > 0.0 ? t2[0] / rho : 0.0;
      rho = t2[0];
      rr = t2[1];
      ++k;
      for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
        const int64_t o = (t % j) + (t / j) * ld;
        Xn[o] = fma(beta, ldcg(X + o), a.zb[o]);
      }
      if (!grid_barrier(a)) goto timeout;
      double* tmp = X;
      X = Xn;
      Xn = tmp;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = (double)k;
    a.out[1] = rr;
    a.out[2] = (double)status;
  }
  return;
timeout:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = (double)k;
    a.out[1] = rr;
    a.out[2] = 3.0;
  }
}

}  // namespace

int galerkin_grid_size() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, galerkin_cg_kernel, kGThreads, 0) != cudaSuccess || per < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

cudaError_t galerkin_cg_launch(int nb, int j, int m, int64_t ld, double lam, const double* A1, const double* A2,
                               const double* B1, const double* B2, const double* G, const double* H,
                               const double* F, const double* Dg, double* Z, double* R, double* Pa, double* Pb,
                               double* Q, double* T2, double* T1, double* TH, double* Gw, double* zb, double* part,
                               unsigned* bar, int* err, double tol2, int maxit, double* out, cudaStream_t st) {
  GalArgs a{};
  a.j = j;
  a.m = m;
  a.nb = nb;
  a.ld = ld;
  a.lam = lam;
  a.A1 = A1;
  a.A2 = A2;
  a.B1 = B1;
  a.B2 = B2;
  a.G = G;
  a.H = H;
  a.F = F;
  a.Dg = Dg;
  a.Z = Z;
  a.R = R;
  a.Pa = Pa;
  a.Pb = Pb;
  a.Q = Q;
  a.T2 = T2;
  a.T1 = T1;
  a.TH = TH;
  a.Gw = Gw;
  a.zb = zb;
  a.part = part;
  a.bar = bar;
  a.err = err;
  a.tol2 = tol2;
  a.maxit = maxit;
  a.out = out;
  void* args[] = {&a};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)galerkin_cg_kernel, dim3(nb), dim3(kGThreads), args, 0, st);
}

}  // namespace cr
