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
// Eigenbasis form (fast diagonalization).  With A1 = Qa diag(la) Qa^T and
// B1 = Qb diag(lb) Qb^T (A1 = U^T L_y U, B1 = V^T L_x V), the CG runs on
// Zt = Qa^T Z Qb, where the operator is
//   Kt(X) = lam (X B2t + 2 diag(la) X diag(lb) + A2t X) + Qa^T [G_a Qa X ht_a] ht_a^T
// with A2t = Qa^T A2 Qa, B2t = Qb^T B2 Qb, ht_a = Qb^T h_a: the A1 X B1 product
// becomes a scaling, two of the four j^3 products per iteration go, and the data
// term needs two thin (j x m) products more:
//   A  T2 = X B2t, TH = X Ht
//   A' Y = Qa TH
//   B  Gw(:, a) = G_a Y(:, a)
//   B' Gt = Qa^T Gw
//   C  Q = lam T2 + 2 lam la_i lb_l X + lam A2t X + Gt Ht^T
// Dg then holds the diagonal of Kt with the data term's G_a replaced by its mean
// diagonal g_a (an SPD preconditioner; the iterate it converges to is the same).
// With that replacement the data term of row i of Kt is Zt(i, :) Hg Hg^T
// (Hg = Ht diag(sqrt g), rank m), so row i of the operator's "diagonal part" is
// D_i + Hg Hg^T with D_i = diag(Dl(i, :)): the row-wise Sherman-Morrison-Woodbury
// preconditioner inverts exactly that (m x m capacitance matrix C_i per row,
// inverted once per projection) at the cost of two thin products per iteration:
//   D  ... R -= alpha Q; y = R ./ Dl
//   S  S(i, :) = C_i^-1 (y(i, :) Hg)           (one CTA per row)
//   Z  z = y - (S Hg^T) ./ Dl, <R, z>, <R, R>    (8x8 tiles)
// Tiles use all CTAs; each output is summed in a fixed order (k split in four
// fixed ranges added in order), and every CTA adds the per-CTA partial sums of
// the inner products in block order, so all CTAs take the same decisions and
// the result is bitwise reproducible.  Data produced by other CTAs in the same
// launch is read with ld.global.cg (L2), never from a possibly stale L1 line.
// The grid barrier spins with a bound; on timeout it raises an error word that
// makes every CTA leave, and the host reports CR_ETIMEOUT.
#include <algorithm>

#include "cr_common.cuh"

namespace cr {

namespace {

constexpr int kGThreads = 256;
constexpr int TS = 8;

template <class T>
struct GalArgs {
  int j, m, nb;
  int64_t ld;
  double lam;
  const T *A1, *A2, *B1, *B2, *G, *H, *F, *Dg;
  T *Z, *R, *Pa, *Pb, *Q, *T2, *T1, *TH, *Gw, *zb;
  double* part;        // [nb * 4]
  unsigned* bar;       // [0] arrivals, [1] generation
  int* err;            // timeout flag
  double tol2;         // stop when |R|^2 <= tol2
  int maxit;
  double* out;         // [0] iterations, [1] |R|^2, [2] status (0 ok, 1 cap, 2 breakdown, 3 barrier timeout)
  // eigenbasis form (Qa == nullptr: the original basis); A1, B1 unused there
  const T *Qa, *la, *lb;
  T *Yb, *Gt;  // ld x m work
  // row-wise Sherman-Morrison-Woodbury preconditioner (Ci == nullptr: z = R ./ Dg):
  //   row i of z = D_i^-1 r_i - D_i^-1 Hg C_i^-1 Hg^T D_i^-1 r_i,  D_i = Dl(i, :)
  // kept in float64 in both instantiations: where the data term dominates a row, the
  // correction cancels most of D_i^-1 r_i, which float32 would not resolve
  const double *Dl, *Hg, *Ci;  // j x j (ld), ld x m, j blocks of m x m
  double *Sb, *Yd;             // ld x m, j x j (ld) work
  T* Zz;                       // j x j (ld) work
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// Grid-wide barrier with a bounded spin.  Returns false if the error word is set.
template <class T>
__device__ __forceinline__ bool grid_barrier(const GalArgs<T>& a) {
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
template <int NV, class T>
__device__ void cta_partial(double (&v)[NV], const GalArgs<T>& a) {
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
template <int NV, class T>
__device__ void grid_total(const GalArgs<T>& a, double (&out)[NV]) {
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
// Staging tiles of tile_term: one buffer per element type, shared by every
// instantiation (each lambda pair would otherwise declare its own arrays).
template <class T>
__device__ __forceinline__ T (*tile_buf())[TS + 1] {
  __shared__ T buf[64][TS + 1];
  return buf;
}

template <class T, class GA, class GB>
__device__ __forceinline__ T tile_term(int i0, int l0, int M, int N, int K, GA ga, GB gb, T acc) {
  T(*As)[TS + 1] = tile_buf<T>();
  T(*Bs)[TS + 1] = As + 32;
  const int tid = threadIdx.x;
  const int o = tid & 63, g = tid >> 6;
  const int oi = o & 7, ol = o >> 3;
  for (int k0 = 0; k0 < K; k0 += 32) {
    {
      const int ii = tid & 7, kk = tid >> 3;
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < M && k < K) ? ga(i, k) : (T)0;
    }
    {
      const int kk = tid & 31, ll = tid >> 5;
      const int l = l0 + ll, k = k0 + kk;
      Bs[kk][ll] = (l < N && k < K) ? gb(k, l) : (T)0;
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
template <class T>
__device__ __forceinline__ T tile_reduce(T acc, bool& valid) {
  __shared__ T red[4][64];
  const int tid = threadIdx.x;
  red[tid >> 6][tid & 63] = acc;
  __syncthreads();
  T v = (T)0;
  valid = tid < 64;
  if (valid) v = ((red[0][tid] + red[1][tid]) + red[2][tid]) + red[3][tid];
  __syncthreads();
  return v;
}

// K(X) -> Q for X = Xin (phases A, B, C; A' and B' in the eigenbasis form);
// returns <X, Q> partial of this CTA in pq.
template <class T>
__device__ bool apply_K(const GalArgs<T>& a, const T* X, double& pq) {
  const int j = a.j, m = a.m;
  const int64_t ld = a.ld;
  const int nt = (j + TS - 1) / TS, ntm = (m + TS - 1) / TS;
  const bool eig = a.Qa != nullptr;
  // A
  const int nA = eig ? 1 : 2;
  const int itemsA = nA * nt * nt + nt * ntm;
  for (int it = blockIdx.x; it < itemsA; it += a.nb) {
    int which, ti, tl;
    if (it < nt * nt) {
      which = 0; ti = it % nt; tl = it / nt;
    } else if (it < nA * nt * nt) {
      which = 1; ti = (it - nt * nt) % nt; tl = (it - nt * nt) / nt;
    } else {
      which = 2; ti = (it - nA * nt * nt) % nt; tl = (it - nA * nt * nt) / nt;
    }
    const int N = which == 2 ? m : j;
    const T* Bm = which == 0 ? a.B2 : which == 1 ? a.B1 : a.H;
    T* out = which == 0 ? a.T2 : which == 1 ? a.T1 : a.TH;
    T acc = tile_term<T>(ti * TS, tl * TS, j, N, j, [&](int i, int k) { return ldcg(X + i + k * ld); },
                         [&](int k, int l) { return Bm[k + l * ld]; }, (T)0);
    bool v;
    const T r = tile_reduce<T>(acc, v);
    if (v) {
      const int i = ti * TS + (threadIdx.x & 7), l = tl * TS + (threadIdx.x >> 3);
      if (i < j && l < N) out[i + l * ld] = r;
    }
  }
  if (!grid_barrier(a)) return false;
  // A' (eigenbasis): Y = Qa TH
  if (eig) {
    for (int it = blockIdx.x; it < nt * ntm; it += a.nb) {
      const int ti = it % nt, tl = it / nt;
      T acc = tile_term<T>(ti * TS, tl * TS, j, m, j, [&](int i, int k) { return a.Qa[i + k * ld]; },
                           [&](int k, int l) { return ldcg(a.TH + k + l * ld); }, (T)0);
      bool v;
      const T r = tile_reduce<T>(acc, v);
      if (v) {
        const int i = ti * TS + (threadIdx.x & 7), l = tl * TS + (threadIdx.x >> 3);
        if (i < j && l < m) a.Yb[i + l * ld] = r;
      }
    }
    if (!grid_barrier(a)) return false;
  }
  // B
  const T* src = eig ? a.Yb : a.TH;
  const int nr = (j + 63) / 64;
  for (int it = blockIdx.x; it < m * nr; it += a.nb) {
    const int al = it / nr, rt = it % nr;
    const int i = rt * 64 + (threadIdx.x & 63), g = threadIdx.x >> 6;
    const T* Ga = a.G + (int64_t)al * ld * ld;
    T acc = (T)0;
    if (i < j) {
      const int q0 = g * ((j + 3) / 4), q1 = min(j, q0 + (j + 3) / 4);
      for (int q = q0; q < q1; ++q) acc = fma(Ga[i + q * ld], ldcg(src + q + al * ld), acc);
    }
    __shared__ T rb[4][64];
    rb[g][threadIdx.x & 63] = acc;
    __syncthreads();
    if (threadIdx.x < 64 && i < j)
      a.Gw[i + (int64_t)al * ld] = ((rb[0][threadIdx.x] + rb[1][threadIdx.x]) + rb[2][threadIdx.x]) + rb[3][threadIdx.x];
    __syncthreads();
  }
  if (!grid_barrier(a)) return false;
  // B' (eigenbasis): Gt = Qa^T Gw
  if (eig) {
    for (int it = blockIdx.x; it < nt * ntm; it += a.nb) {
      const int ti = it % nt, tl = it / nt;
      T acc = tile_term<T>(ti * TS, tl * TS, j, m, j, [&](int i, int k) { return a.Qa[k + i * ld]; },
                           [&](int k, int l) { return ldcg(a.Gw + k + l * ld); }, (T)0);
      bool v;
      const T r = tile_reduce<T>(acc, v);
      if (v) {
        const int i = ti * TS + (threadIdx.x & 7), l = tl * TS + (threadIdx.x >> 3);
        if (i < j && l < m) a.Gt[i + l * ld] = r;
      }
    }
    if (!grid_barrier(a)) return false;
  }
  // C
  const T* gdat = eig ? a.Gt : a.Gw;
  double dotpq = 0.0;
  const T lam = (T)a.lam;
  const T lam2 = (T)(2.0 * a.lam);
  for (int it = blockIdx.x; it < nt * nt; it += a.nb) {
    const int ti = it % nt, tl = it / nt;
    const int i0 = ti * TS, l0 = tl * TS;
    T acc = (T)0;
    if (!eig)
      acc = tile_term<T>(i0, l0, j, j, j, [&](int i, int k) { return lam2 * a.A1[i + k * ld]; },
                         [&](int k, int l) { return ldcg(a.T1 + k + l * ld); }, acc);
    acc = tile_term<T>(i0, l0, j, j, j, [&](int i, int k) { return lam * a.A2[i + k * ld]; },
                       [&](int k, int l) { return ldcg(X + k + l * ld); }, acc);
    acc = tile_term<T>(i0, l0, j, j, m, [&](int i, int k) { return ldcg(gdat + i + k * ld); },
                       [&](int k, int l) { return a.H[l + k * ld]; }, acc);
    bool v;
    const T r = tile_reduce<T>(acc, v);
    if (v) {
      const int i = i0 + (threadIdx.x & 7), l = l0 + (threadIdx.x >> 3);
      if (i < j && l < j) {
        const int64_t o = i + l * ld;
        const T x = ldcg(X + o);
        T q = fma(lam, ldcg(a.T2 + o), r);
        if (eig) q = fma(lam2 * a.la[i] * a.lb[l], x, q);
        a.Q[o] = q;
        dotpq += (double)x * (double)q;
      }
    }
  }
  pq = dotpq;
  return true;
}

// Row-wise SMW preconditioner, after y = R ./ Dl has been stored in Yz (and a grid
// barrier): S(i, :) = C_i^-1 (y_i Hg) per row, then z = y - (S Hg^T) ./ Dl into Zo
// with this CTA's partials of <R, z> and <R, R> in v.
template <class T>
__device__ bool precond_smw(const GalArgs<T>& a, const double* Yz, T* Zo, double (&v)[2]) {
  const int j = a.j, m = a.m;
  const int64_t ld = a.ld;
  __shared__ double wpart[8][128];
  __shared__ double wrow[128];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;  // 8 groups of 32
  const int kc = (j + 7) / 8, k0 = min(j, grp * kc), k1 = min(j, k0 + kc);
  for (int i = blockIdx.x; i < j; i += a.nb) {
    for (int al = lane; al < m; al += 32) {
      double s = 0.0;
      for (int k = k0; k < k1; ++k) s = fma(ldcg(Yz + i + k * ld), a.Hg[k + al * ld], s);
      wpart[grp][al] = s;
    }
    __syncthreads();
    if (threadIdx.x < m) {
      double s = 0.0;
#pragma unroll
      for (int g = 0; g < 8; ++g) s += wpart[g][threadIdx.x];
      wrow[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < m) {
      const double* c = a.Ci + ((int64_t)i * m + threadIdx.x) * m;
      double s = 0.0;
      for (int b = 0; b < m; ++b) s = fma(c[b], wrow[b], s);
      a.Sb[i + threadIdx.x * ld] = s;
    }
    __syncthreads();
  }
  if (!grid_barrier(a)) return false;
  const int nt = (j + TS - 1) / TS;
  v[0] = v[1] = 0.0;
  for (int it = blockIdx.x; it < nt * nt; it += a.nb) {
    const int ti = it % nt, tl = it / nt;
    double acc = tile_term<double>(ti * TS, tl * TS, j, j, m, [&](int i, int k) { return ldcg(a.Sb + i + k * ld); },
                                   [&](int k, int l) { return a.Hg[l + k * ld]; }, 0.0);
    bool ok;
    const double r = tile_reduce<double>(acc, ok);
    if (ok) {
      const int i = ti * TS + (threadIdx.x & 7), l = tl * TS + (threadIdx.x >> 3);
      if (i < j && l < j) {
        const int64_t o = i + l * ld;
        const T z = (T)(ldcg(Yz + o) - r / a.Dl[o]);
        const T rv = ldcg(a.R + o);
        Zo[o] = z;
        v[0] += (double)rv * (double)z;
        v[1] += (double)rv * (double)rv;
      }
    }
  }
  return true;
}

template <class T>
__global__ void __launch_bounds__(kGThreads, 1) galerkin_cg_kernel(const GalArgs<T> a) {
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
  if (a.Ci) {
    for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
      const int64_t o = (t % j) + (t / j) * ld;
      const T r = a.F[o] - ldcg(a.Q + o);
      a.R[o] = r;
      a.Yd[o] = (double)r / a.Dl[o];
    }
    if (!grid_barrier(a)) goto timeout;
    double v[2];
    if (!precond_smw(a, a.Yd, a.Pa, v)) goto timeout;
    cta_partial<2>(v, a);
  } else {
    double v[2] = {0.0, 0.0};
    for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
      const int64_t o = (t % j) + (t / j) * ld;
      const T r = a.F[o] - ldcg(a.Q + o);
      const T z = r / a.Dg[o];
      a.R[o] = r;
      a.Pa[o] = z;
      v[0] += (double)r * (double)z;
      v[1] += (double)r * (double)r;
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
    T* X = a.Pa;
    T* Xn = a.Pb;
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
      const T alpha = (T)(rho / pqt[0]);
      if (a.Ci) {
        for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
          const int64_t o = (t % j) + (t / j) * ld;
          a.Z[o] = fma(alpha, ldcg(X + o), a.Z[o]);
          const T r = fma(-alpha, ldcg(a.Q + o), a.R[o]);
          a.R[o] = r;
          a.Yd[o] = (double)r / a.Dl[o];
        }
        if (!grid_barrier(a)) goto timeout;
        double v[2];
        if (!precond_smw(a, a.Yd, a.Zz, v)) goto timeout;
        cta_partial<2>(v, a);
      } else {
        double v[2] = {0.0, 0.0};
        for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
          const int64_t o = (t % j) + (t / j) * ld;
          a.Z[o] = fma(alpha, ldcg(X + o), a.Z[o]);
          const T r = fma(-alpha, ldcg(a.Q + o), a.R[o]);
          a.R[o] = r;
          const T z = r / a.Dg[o];
          a.zb[o] = z;
          v[0] += (double)r * (double)z;
          v[1] += (double)r * (double)r;
        }
        cta_partial<2>(v, a);
      }
      if (!grid_barrier(a)) goto timeout;
      double t2[2];
      grid_total<2>(a, t2);
      const T beta = (T)(rho > 0.0 ? t2[0] / rho : 0.0);
      rho = t2[0];
      rr = t2[1];
      ++k;
      for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
        const int64_t o = (t % j) + (t / j) * ld;
        Xn[o] = fma(beta, ldcg(X + o), a.Ci ? ldcg(a.Zz + o) : a.zb[o]);
      }
      if (!grid_barrier(a)) goto timeout;
      T* tmp = X;
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

namespace {
// g_a = tr(G_a) / j, one CTA per a
__global__ void gal_trace_kernel(int j, int64_t ld, const double* __restrict__ G, double* __restrict__ g) {
  const double* Ga = G + (int64_t)blockIdx.x * ld * ld;
  double s = 0.0;
  for (int i = threadIdx.x; i < j; i += blockDim.x) s += Ga[i + (int64_t)i * ld];
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g[blockIdx.x] = t / (double)j;
  }
}

// Dl(i, k) = lam (A2t_ii + 2 la_i lb_k + B2t_kk), Den = Dl + sum_a g_a Ht(k, a)^2,
// and (first column of threads) Hg(k, a) = sqrt(g_a) Ht(k, a)
__global__ void gal_eig_den_kernel(int j, int m, int64_t ld, double lam, const double* __restrict__ A2t,
                                   const double* __restrict__ B2t, const double* __restrict__ la,
                                   const double* __restrict__ lb, const double* __restrict__ g,
                                   const double* __restrict__ Ht, double* __restrict__ Den, double* __restrict__ Dl,
                                   double* __restrict__ Hg) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)j * j) return;
  const int i = (int)(t % j), k = (int)(t / j);
  double h = 0.0;
  for (int a = 0; a < m; ++a) {
    const double x = Ht[k + (int64_t)a * ld];
    h = fma(g[a] * x, x, h);
    if (i == 0) Hg[k + (int64_t)a * ld] = sqrt(fmax(g[a], 0.0)) * x;
  }
  const double li = fmax(la[i], 0.0), lk = fmax(lb[k], 0.0);  // A1, B1 are positive semidefinite
  const double dl = lam * (A2t[i + (int64_t)i * ld] + 2.0 * li * lk + B2t[k + (int64_t)k * ld]);
  Dl[i + (int64_t)k * ld] = dl;
  Den[i + (int64_t)k * ld] = dl + h;
}

// C_i = I + Hg^T diag(1 / Dl(i, :)) Hg (m x m, SPD with eigenvalues >= 1), inverted in
// shared memory by Gauss-Jordan elimination without pivoting; one CTA per row i.
__global__ void gal_smw_setup_kernel(int j, int m, int64_t ld, const double* __restrict__ Dl,
                                     const double* __restrict__ Hg, double* __restrict__ Ci) {
  extern __shared__ double sm[];
  double* C = sm;              // m x m, row-major
  double* prow = C + m * m;    // scaled pivot row
  double* fcol = prow + m;     // pivot column
  double* dinv = fcol + m;     // 1 / Dl(i, :)
  const int i = blockIdx.x;
  for (int k = threadIdx.x; k < j; k += blockDim.x) dinv[k] = 1.0 / Dl[i + (int64_t)k * ld];
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int r = t / m, c = t % m;
    if (c < r) continue;
    const double* hr = Hg + (int64_t)r * ld;
    const double* hc = Hg + (int64_t)c * ld;
    double s = 0.0;
    for (int k = 0; k < j; ++k) s = fma(hr[k] * dinv[k], hc[k], s);
    s += r == c ? 1.0 : 0.0;
    C[r * m + c] = s;
    C[c * m + r] = s;
  }
  for (int p = 0; p < m; ++p) {
    __syncthreads();
    const double piv = 1.0 / C[p * m + p];
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      prow[t] = (t == p ? 1.0 : C[p * m + t]) * piv;
      fcol[t] = C[t * m + p];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int r = t / m, c = t % m;
      C[t] = r == p ? prow[c] : (c == p ? 0.0 : C[t]) - fcol[r] * prow[c];
    }
  }
  __syncthreads();
  double* out = Ci + (int64_t)i * m * m;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) out[t] = C[t];
}
}  // namespace

void galerkin_eig_diag(int j, int m, int64_t ld, double lam, const double* A2t, const double* B2t, const double* la,
                       const double* lb, const double* G, const double* Ht, double* g, double* Den, double* Dl,
                       double* Hg, cudaStream_t st) {
  if (j <= 0) return;
  if (m > 0) {
    count_launch();
    gal_trace_kernel<<<m, 256, 0, st>>>(j, ld, G, g);
  }
  const int64_t tot = (int64_t)j * j;
  count_launch();
  gal_eig_den_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(j, m, ld, lam, A2t, B2t, la, lb, g, Ht, Den,
                                                                       Dl, Hg);
}

size_t galerkin_smw_smem(int j, int m) { return sizeof(double) * ((size_t)m * m + 2 * (size_t)m + (size_t)j); }

cudaError_t galerkin_smw_setup(int j, int m, int64_t ld, const double* Dl, const double* Hg, double* Ci,
                               cudaStream_t st) {
  if (j <= 0 || m <= 0) return cudaSuccess;
  if (m > 128) return cudaErrorNotSupported;
  const size_t smem = galerkin_smw_smem(j, m);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(gal_smw_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  gal_smw_setup_kernel<<<j, 256, smem, st>>>(j, m, ld, Dl, Hg, Ci);
  return cudaGetLastError();
}

int galerkin_grid_size() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, galerkin_cg_kernel<double>, kGThreads, 0) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

template <class T>
cudaError_t galerkin_cg_launch(int nb, int j, int m, int64_t ld, double lam, const T* A1, const T* A2, const T* B1,
                               const T* B2, const T* G, const T* H, const T* F, const T* Dg, T* Z, T* R, T* Pa,
                               T* Pb, T* Q, T* T2, T* T1, T* TH, T* Gw, T* zb, double* part, unsigned* bar,
                               int* err, double tol2, int maxit, double* out, cudaStream_t st, const GalEig<T>* eig) {
  GalArgs<T> a{};
  if (eig) {
    a.Qa = eig->Qa;
    a.la = eig->la;
    a.lb = eig->lb;
    a.Yb = eig->Y;
    a.Gt = eig->Gt;
    if (eig->Ci && m <= 128) {
      a.Dl = eig->Dl;
      a.Hg = eig->Hg;
      a.Ci = eig->Ci;
      a.Sb = eig->S;
      a.Yd = eig->Yd;
      a.Zz = eig->Zz;
    }
  }
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
  return cudaLaunchCooperativeKernel((const void*)galerkin_cg_kernel<T>, dim3(nb), dim3(kGThreads), args, 0, st);
}

template cudaError_t galerkin_cg_launch<double>(int, int, int, int64_t, double, const double*, const double*,
                                                const double*, const double*, const double*, const double*,
                                                const double*, const double*, double*, double*, double*, double*,
                                                double*, double*, double*, double*, double*, double*, double*,
                                                unsigned*, int*, double, int, double*, cudaStream_t,
                                                const GalEig<double>*);
template cudaError_t galerkin_cg_launch<float>(int, int, int, int64_t, double, const float*, const float*,
                                               const float*, const float*, const float*, const float*, const float*,
                                               const float*, float*, float*, float*, float*, float*, float*, float*,
                                               float*, float*, float*, double*, unsigned*, int*, double, int, double*,
                                               cudaStream_t, const GalEig<float>*);

}  // namespace cr

// ---------------------------------------------------------------------------
// Single-cluster float32 Galerkin CG for the inner solves of the mixed form
// (j <= 128, m <= 128), in the original basis or the eigenbasis form (then
// TH(:, own a) goes through Y = Qa TH before G_a and the result through Qa^T,
// both local to the CTA that owns a, and the A1 X B1 term is a scaling).  The columns of the CG matrices are split over the
// CTAs of one cluster; every CTA keeps a full copy of the current search
// direction X and of Gw = [G_a X h_a]_a in shared memory, refreshed by an
// all-gather over distributed shared memory, so every product is local:
//   T2 = X B2(:, own), T1 = X B1(:, own), TH = X H(:, own a), Gw(:, own a) = G_a TH(:, a)
//   Q(:, own) = lam T2 + 2 lam A1 T1 + lam A2 X(:, own) + Gw H(own, :)^T
// Inner products and CG scalars are double-float (cr_df.cuh), reduced in a
// fixed order (threads, warps, CTAs in rank order).  Four cluster barriers
// per iteration, no grid barrier, no launch.
#include <cooperative_groups.h>

#include "cr_df.cuh"

namespace cr {
namespace {

namespace cgc = cooperative_groups;

constexpr int kClThreads = 512;
constexpr int kClMax = 16;

struct GalClArgs {
  int j, m, cw, aw;  // rank, injections, columns per CTA, injections per CTA
  int64_t ld;
  float lam;
  const float *A1, *A2, *B1, *B2, *G, *H, *F, *Dg;
  const float *Qa, *la, *lb;  // eigenbasis form (Qa == nullptr: the original basis)
  float* Z;
  float tol2;  // stop when |R|^2 <= tol2
  int maxit;
  double* out;
};

__device__ __forceinline__ DF cl_block_df(DF v, DF* scr) {
  // returns the CTA sum (valid in thread 0)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_df(v);
  if (lane == 0) scr[wid] = v;
  __syncthreads();
  DF t{0.f, 0.f};
  if (wid == 0) {
    t = lane < nw ? scr[lane] : DF{0.f, 0.f};
    t = warp_sum_df(t);
  }
  __syncthreads();
  return t;
}

// Copy into buf every element whose block (of `bw` consecutive elements) is
// owned by another CTA, from that CTA's buf.  Eight independent loads are
// issued per thread before their stores, so the distributed-shared-memory
// latencies overlap instead of adding up.
__device__ __forceinline__ void gather_blocks(cgc::cluster_group& cl, float* buf, int total, int bw, int rank) {
  const int nth = blockDim.x;
  for (int t0 = threadIdx.x; t0 < total; t0 += 8 * nth) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = t0 + u * nth;
      const int owner = idx < total ? idx / bw : rank;
      v[u] = owner != rank ? cl.map_shared_rank(buf, (unsigned)owner)[idx] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = t0 + u * nth;
      if (idx < total && idx / bw != rank) buf[idx] = v[u];
    }
  }
}

__global__ void __launch_bounds__(kClThreads, 1) galerkin_cluster_f32_kernel(const GalClArgs a) {
  // Chronopoulos-Gear form of the Jacobi-preconditioned matrix CG: one
  // operator application (on U = D^-1 R) and one fused reduction of
  // <R, U>, <U, W>, <R, R> per iteration.
  cgc::cluster_group cl = cgc::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int j = a.j, m = a.m, cw = a.cw, aw = a.aw;
  const int64_t ld = a.ld;
  const int c0 = min(j, rank * cw), c1 = min(j, c0 + cw), nc = c1 - c0;
  const int a0 = min(m, rank * aw), a1 = min(m, a0 + aw), na = a1 - a0;
  extern __shared__ __align__(16) float fsm[];
  float* Xf = fsm;                 // j x j (ld j): full copy of U
  float* Gwf = Xf + j * j;         // j x m (ld j)
  float* Zo = Gwf + j * m;         // own blocks, j x cw each (ld j)
  float* Ro = Zo + j * cw;
  float* Po = Ro + j * cw;
  float* So = Po + j * cw;
  float* Wo = So + j * cw;
  float* T1o = Wo + j * cw;
  float* T2o = T1o + j * cw;
  float* Dio = T2o + j * cw;       // 1 / diag(K) on own columns
  float* THo = Dio + j * cw;       // j x aw
  float* Yo = THo + j * aw;        // j x aw (eigenbasis form: Qa TH)
  DF* scr = reinterpret_cast<DF*>(Yo + j * aw);  // [32]
  DF* red = scr + 32;              // [4]
  float* scal = reinterpret_cast<float*>(red + 4);  // [8]
  float* Uo = Xf + (int64_t)c0 * j;  // own columns of U inside the full copy
  const int tid = threadIdx.x, nth = blockDim.x;
  const float lam = a.lam, lam2 = 2.f * a.lam;
  const bool eig = a.Qa != nullptr;

  // Z = 0, R = F, U = D^-1 R
  for (int t = tid; t < j * nc; t += nth) {
    const int i = t % j, lc = t / j;
    const int64_t o = i + (int64_t)(c0 + lc) * ld;
    const float r = a.F[o], di = 1.f / a.Dg[o];
    Zo[t] = 0.f;
    Ro[t] = r;
    Dio[t] = di;
    Uo[t] = r * di;
    Po[t] = 0.f;
    So[t] = 0.f;
  }
  int it = 0, status = 0;
  DF gam_prev{1.f, 0.f}, alpha_prev{1.f, 0.f}, rrt{0.f, 0.f};
  for (;;) {
    cl.sync();  // B1: own columns of U published
    gather_blocks(cl, Xf, j * j, j * cw, rank);
    __syncthreads();
    if (eig) {
      for (int t = tid; t < j * nc; t += nth) {
        const int i = t % j, lc = t / j;
        const float* b2 = a.B2 + (int64_t)(c0 + lc) * ld;
        float s2 = 0.f;
        for (int k = 0; k < j; ++k) s2 = fmaf(Xf[i + k * j], __ldg(b2 + k), s2);
        T2o[t] = s2;
      }
    } else {
      for (int t = tid; t < j * nc; t += nth) {
        const int i = t % j, lc = t / j;
        const float* b2 = a.B2 + (int64_t)(c0 + lc) * ld;
        const float* b1 = a.B1 + (int64_t)(c0 + lc) * ld;
        float s2 = 0.f, s1 = 0.f;
        for (int k = 0; k < j; ++k) {
          const float x = Xf[i + k * j];
          s2 = fmaf(x, __ldg(b2 + k), s2);
          s1 = fmaf(x, __ldg(b1 + k), s1);
        }
        T2o[t] = s2;
        T1o[t] = s1;
      }
    }
    for (int t = tid; t < j * na; t += nth) {
      const int i = t % j, la = t / j;
      const float* h = a.H + (int64_t)(a0 + la) * ld;
      float s = 0.f;
      for (int k = 0; k < j; ++k) s = fmaf(Xf[i + k * j], __ldg(h + k), s);
      THo[t] = s;
    }
    __syncthreads();
    if (eig) {  // Y = Qa TH on own injections
      for (int t = tid; t < j * na; t += nth) {
        const int i = t % j, la = t / j;
        float s = 0.f;
        for (int k = 0; k < j; ++k) s = fmaf(__ldg(a.Qa + i + (int64_t)k * ld), THo[k + la * j], s);
        Yo[t] = s;
      }
      __syncthreads();
    }
    const float* src = eig ? Yo : THo;
    for (int t = tid; t < j * na; t += nth) {
      const int i = t % j, la = t / j;
      const float* g = a.G + (int64_t)(a0 + la) * ld * ld;
      float s = 0.f;
      for (int q = 0; q < j; ++q) s = fmaf(__ldg(g + i + (int64_t)q * ld), src[q + la * j], s);
      Gwf[i + (a0 + la) * j] = s;
    }
    if (eig) {  // Gw <- Qa^T Gw on own injections (through TH)
      __syncthreads();
      for (int t = tid; t < j * na; t += nth) {
        const int i = t % j, la = t / j;
        const float* q = a.Qa + (int64_t)i * ld;
        float s = 0.f;
        for (int k = 0; k < j; ++k) s = fmaf(__ldg(q + k), Gwf[k + (a0 + la) * j], s);
        THo[t] = s;
      }
      __syncthreads();
      for (int t = tid; t < j * na; t += nth) {
        const int i = t % j, la = t / j;
        Gwf[i + (a0 + la) * j] = THo[t];
      }
    }
    cl.sync();  // B2: own columns of Gw published
    gather_blocks(cl, Gwf, j * m, j * aw, rank);
    __syncthreads();
    // W = K(U) on own columns; partial <R, U>, <U, W>, <R, R>
    DF v0{0.f, 0.f}, v1{0.f, 0.f}, v2{0.f, 0.f};
    for (int t = tid; t < j * nc; t += nth) {
      const int i = t % j, lc = t / j;
      const int l = c0 + lc;
      float s1 = 0.f, s2 = 0.f, s3 = 0.f;
      if (eig) {
        for (int k = 0; k < j; ++k) s2 = fmaf(__ldg(a.A2 + i + (int64_t)k * ld), Uo[k + lc * j], s2);
        s1 = __ldg(a.la + i) * __ldg(a.lb + l) * Uo[t];
      } else {
        for (int k = 0; k < j; ++k) {
          s1 = fmaf(__ldg(a.A1 + i + (int64_t)k * ld), T1o[k + lc * j], s1);
          s2 = fmaf(__ldg(a.A2 + i + (int64_t)k * ld), Uo[k + lc * j], s2);
        }
      }
      for (int al = 0; al < m; ++al) s3 = fmaf(Gwf[i + al * j], __ldg(a.H + l + (int64_t)al * ld), s3);
      const float w = lam * T2o[t] + lam2 * s1 + lam * s2 + s3;
      Wo[t] = w;
      const float u = Uo[t], r = Ro[t];
      v0 = df_add(v0, df_prod(r, u));
      v1 = df_add(v1, df_prod(u, w));
      v2 = df_add(v2, df_prod(r, r));
    }
    {
      const DF s0 = cl_block_df(v0, scr);
      const DF s1 = cl_block_df(v1, scr);
      const DF s2 = cl_block_df(v2, scr);
      if (tid == 0) {
        red[0] = s0;
        red[1] = s1;
        red[2] = s2;
      }
    }
    cl.sync();  // B3
    if (tid < 32) {
      DF g{0.f, 0.f}, dl{0.f, 0.f}, rh{0.f, 0.f};
      if (tid < C) {
        const DF* rm = cl.map_shared_rank(red, tid);
        g = rm[0];
        dl = rm[1];
        rh = rm[2];
      }
      g = warp_sum_df(g);
      dl = warp_sum_df(dl);
      rh = warp_sum_df(rh);
      if (tid == 0) {
        float flag = 0.f;
        DF alpha{0.f, 0.f}, beta{0.f, 0.f};
        if (rh.hi <= a.tol2) {
          flag = 1.f;
        } else if (it >= a.maxit) {
          flag = 2.f;
        } else {
          DF den = dl;
          if (it > 0) {
            beta = df_div(g, gam_prev);
            den = df_sub(dl, df_div(df_mul(beta, g), alpha_prev));
          }
          if (!(den.hi > 0.f) || !isfinite(den.hi)) {
            flag = 3.f;
          } else {
            alpha = df_div(g, den);
            gam_prev = g;
            alpha_prev = alpha;
          }
        }
        scal[0] = flag;
        scal[1] = alpha.hi;
        scal[2] = beta.hi;
        reinterpret_cast<DF*>(scal)[2] = rh;
      }
    }
    __syncthreads();
    const float flag = scal[0];
    rrt = reinterpret_cast<DF*>(scal)[2];
    if (flag == 1.f) break;
    if (flag == 2.f) {
      status = 1;
      break;
    }
    if (flag == 3.f) {
      status = 2;
      break;
    }
    const float alpha = scal[1], beta = scal[2];
    for (int t = tid; t < j * nc; t += nth) {
      const float p = fmaf(beta, Po[t], Uo[t]);
      const float s = fmaf(beta, So[t], Wo[t]);
      Po[t] = p;
      So[t] = s;
      Zo[t] = fmaf(alpha, p, Zo[t]);
      const float r = fmaf(-alpha, s, Ro[t]);
      Ro[t] = r;
      Uo[t] = r * Dio[t];
    }
    ++it;
  }
  for (int t = tid; t < j * nc; t += nth) {
    const int i = t % j, lc = t / j;
    a.Z[i + (int64_t)(c0 + lc) * ld] = Zo[t];
  }
  cl.sync();  // no CTA leaves while another may read its shared memory
  if (rank == 0 && tid == 0) {
    a.out[0] = (double)it;
    a.out[1] = (double)rrt.hi + (double)rrt.lo;
    a.out[2] = (double)status;
  }
}

size_t gal_cl_smem(int j, int m, int cw, int aw) {
  return sizeof(float) * ((size_t)j * j + (size_t)j * m + 9 * (size_t)j * cw + 2 * (size_t)j * aw) +
         sizeof(DF) * 40 + sizeof(float) * 8 + 64;
}

}  // namespace

// Launch the single-cluster float32 Galerkin CG if it fits (j <= 128, m <= 128);
// returns cudaErrorNotSupported otherwise.
cudaError_t galerkin_cluster_f32_launch(int j, int m, int64_t ld, double lam, const float* A1, const float* A2,
                                        const float* B1, const float* B2, const float* G, const float* H,
                                        const float* F, const float* Dg, float* Z, double tol2, int maxit,
                                        double* out, cudaStream_t st, const GalEig<float>* eig) {
  if (j < 1 || j > 128 || m > 128) return cudaErrorNotSupported;
  const int C = std::min(kClMax, j);
  const int cw = (j + C - 1) / C, aw = (m + C - 1) / C;
  const size_t smem = gal_cl_smem(j, m, cw, aw);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(galerkin_cluster_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(galerkin_cluster_f32_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  GalClArgs a{};
  a.j = j;
  a.m = m;
  a.cw = cw;
  a.aw = aw;
  a.ld = ld;
  a.lam = (float)lam;
  a.A1 = A1;
  a.A2 = A2;
  a.B1 = B1;
  a.B2 = B2;
  a.G = G;
  a.H = H;
  a.F = F;
  a.Dg = Dg;
  if (eig) {
    a.Qa = eig->Qa;
    a.la = eig->la;
    a.lb = eig->lb;
  }
  a.Z = Z;
  a.tol2 = (float)tol2;
  a.maxit = maxit;
  a.out = out;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, galerkin_cluster_f32_kernel, a);
}

}  // namespace cr
