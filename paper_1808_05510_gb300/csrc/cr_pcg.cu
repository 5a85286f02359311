// Cluster-resident preconditioned CG for the ALS sub-problems (Sec. 2.3,
// Eqs. ALS_linsys and ALS_linsys_v).
//
// Both operators have the form  lam * [(L + c I)^2 + e I] + data:
//   A_hat = lam((v'L_x^2 v) I + 2 (v'L_x v) L_y + L_y^2) + sum_a diag(Omega_a)(v'X_a)^2
//         = lam[(L_y + cI)^2 + (d - c^2) I] + diag(omega_tilde),  c = v'L_x v, d = |L_x v|^2
//   B_hat = lam(L_x^2 + 2 (u'L_y u) L_x + (u'L_y^2 u) I) + sum_a (u'diag(Omega_a)u) X_a X_a'
//         = lam[(L_x + c'I)^2 + (d' - c'^2) I] + X diag(s) X',  c' = u'L_y u, d' = |L_y u|^2
// so one apply is two sparse stencil passes through an intermediate t = (L + cI) p.
//
// Design: one thread-block cluster owns the whole solve.  The rows are split
// into contiguous chunks, one per CTA; the vector being multiplied and the
// intermediate t live in shared memory and neighbours owned by other CTAs are
// read through distributed shared memory.  The iteration is the
// Chronopoulos-Gear form of PCG, whose three inner products (r,u), (u,w),
// (r,r) share one reduction, so an iteration costs three cluster barriers and
// no kernel launch.  Reductions have a fixed order (warp shuffle tree, then
// warps, then CTAs in rank order), so every CTA computes bit-identical scalars
// and takes the same branch; results are reproducible run to run.  The loop
// is bounded by maxit.
#include <cooperative_groups.h>

#include "cr_common.cuh"
#include "cr_df.cuh"

namespace cg = cooperative_groups;

namespace cr {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV per-thread values over the CTA; thread 0 stores the sums in out[].
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scr, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) scr[wid * NV + q] = v[q];
  }
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

// After a cluster barrier: add the NV partials of all CTAs in rank order and
// broadcast them to the CTA through scal[].
template <int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, double* red, double* scal, int csize) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      if (lane < csize) t = cl.map_shared_rank(red, lane)[q];
      t = warp_sum(t);
      if (lane == 0) scal[q] = t;
    }
  }
  __syncthreads();
}

// (L + shift I) applied to row i of a vector held in distributed shared memory.
__device__ __forceinline__ double lap_row_dsm(const DevLap& L, int i, double vi, double shift, double* buf,
                                              cg::cluster_group& cl) {
  double acc = (L.diag[i] + shift) * vi;
  for (int k = 0; k < L.K; ++k) {
    const int q = __ldg(L.nbrp + (size_t)k * L.n + i);
    if (q < 0) continue;
    const double nv = cl.map_shared_rank(buf, (unsigned)(q >> 24))[q & 0xFFFFFF];
    acc += (L.offw ? __ldg(L.offw + (size_t)k * L.n + i) : -1.0) * nv;
  }
  return acc;
}

template <int KIND>
struct Pcg {
  // t = (L + cI) ub on the owned rows; v side: partial X^T ub of the owned rows.
  static __device__ __forceinline__ void phase_t(const PcgArgs& A, cg::cluster_group& cl, int beg, int nloc,
                                                 double c, double* ub, double* tb, double* ypart) {
    for (int li = threadIdx.x; li < nloc; li += blockDim.x) tb[li] = lap_row_dsm(A.L, beg + li, ub[li], c, ub, cl);
    if (KIND == 1) {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const int rank = (int)cl.block_rank();
      for (int a = wid; a < A.m; a += nw) {
        const int p0 = A.X.lx_ptr[rank * A.m + a], p1 = A.X.lx_ptr[rank * A.m + a + 1];
        double acc = 0.0;
        for (int p = p0 + lane; p < p1; p += 32) acc += A.X.lx_val[p] * ub[A.X.lx_row[p]];
        acc = warp_sum(acc);
        if (lane == 0) ypart[a] = acc;
      }
    }
  }
  // v side: y = X^T ub summed over the cluster; sy[a] = s[a] * y[a].
  static __device__ __forceinline__ void gather_y(const PcgArgs& A, cg::cluster_group& cl, double* ypart,
                                                  const double* sS, double* sY) {
    if (KIND == 1) {
      const int C = (int)cl.num_blocks();
      for (int a = threadIdx.x; a < A.m; a += blockDim.x) {
        double t = 0.0;
        for (int r = 0; r < C; ++r) t += cl.map_shared_rank(ypart, (unsigned)r)[a];
        sY[a] = sS[a] * t;
      }
      __syncthreads();
    }
  }
  // w_i = lam[(L + cI) t + e u]_i + data_i
  static __device__ __forceinline__ double row_w(const PcgArgs& A, cg::cluster_group& cl, int i, int li, double c,
                                                 double e, double ui, double* tb, const double* sY) {
    double w = A.lam * (lap_row_dsm(A.L, i, tb[li], c, tb, cl) + e * ui);
    if (KIND == 0) {
      w += A.omt[i] * ui;
    } else {
      for (int p = A.X.xr_ptr[i]; p < A.X.xr_ptr[i + 1]; ++p) w += A.X.xr_val[p] * sY[A.X.xr_col[p]];
    }
    return w;
  }
};

template <int KIND>
__global__ void __launch_bounds__(kPcgThreads, 1) pcg_cluster_kernel(const PcgArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const DevLap& L = A.L;
  const int chunk = L.chunk;
  const int beg = rank * chunk;
  const int nloc = max(0, min(L.n - beg, chunk));
  const int m = A.m;
  extern __shared__ __align__(16) double sm[];
  double* ub0 = sm;
  double* ub1 = sm + chunk;
  double* tb = sm + 2 * chunk;
  double* red = tb + chunk;   // [8]
  double* ypart = red + 8;    // [m]
  double* sS = ypart + m;     // [m]  xi^2 (u side) or s (v side)
  double* sY = sS + m;        // [m]  s * (X^T p) (v side)
  double* scr = sY + m;       // [32 * 4]
  double* scal = scr + 128;   // [8]
  const double lam = A.lam;
  const double c = A.coef[0];
  const double d = A.coef[1];
  const double e = d - c * c;
  using K = Pcg<KIND>;

  for (int a = threadIdx.x; a < m; a += blockDim.x) sS[a] = KIND == 0 ? A.xi[a] * A.xi[a] : A.s[a];
  __syncthreads();
  // data term diagonal, Jacobi preconditioner, initial guess into shared memory
  for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
    const int i = beg + li;
    double dd = lam * (L.l2diag[i] + 2.0 * c * L.diag[i] + d);
    if (KIND == 0) {
      double o = 0.0;
      for (int a = 0; a < m; ++a) o += (double)A.Om[i + (int64_t)a * A.ldo] * sS[a];
      A.omt[i] = o;
      dd += o;
    } else {
      for (int p = A.X.xr_ptr[i]; p < A.X.xr_ptr[i + 1]; ++p) dd += A.X.xr_val[p] * A.X.xr_val[p] * sS[A.X.xr_col[p]];
    }
    A.dinv[i] = dd > 0.0 ? 1.0 / dd : 1.0;
    ub0[li] = A.x[i];
  }
  cl.sync();
  K::phase_t(A, cl, beg, nloc, c, ub0, tb, ypart);
  cl.sync();
  K::gather_y(A, cl, ypart, sS, sY);
  {
    double v[1] = {0.0};
    for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
      const int i = beg + li;
      const double bi = A.b[i];
      A.r[i] = bi - K::row_w(A, cl, i, li, c, e, ub0[li], tb, sY);
      v[0] += bi * bi;
    }
    block_sum<1>(v, scr, red);
  }
  cl.sync();
  cluster_sum<1>(cl, red, scal, C);
  const double bb = scal[0];
  int it = 0, status = 0;
  double rho = 0.0;
  if (bb == 0.0) {
    for (int li = threadIdx.x; li < nloc; li += blockDim.x) A.x[beg + li] = 0.0;
  } else {
    const double tol2 = A.tol * A.tol * bb;
    double gam_prev = 1.0, alpha_prev = 1.0;
    int cur = 1;
    for (;;) {
      double* ub = cur ? ub1 : ub0;
      for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
        const int i = beg + li;
        ub[li] = A.r[i] * A.dinv[i];
      }
      cl.sync();
      K::phase_t(A, cl, beg, nloc, c, ub, tb, ypart);
      cl.sync();
      K::gather_y(A, cl, ypart, sS, sY);
      double v[3] = {0.0, 0.0, 0.0};
      for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
        const int i = beg + li;
        const double ui = ub[li];
        const double wi = K::row_w(A, cl, i, li, c, e, ui, tb, sY);
        const double ri = A.r[i];
        A.w[i] = wi;
        v[0] += ri * ui;
        v[1] += ui * wi;
        v[2] += ri * ri;
      }
      block_sum<3>(v, scr, red);
      cl.sync();
      cluster_sum<3>(cl, red, scal, C);
      const double gam = scal[0], del = scal[1];
      rho = scal[2];
      if (rho <= tol2) break;
      if (it >= A.maxit) { status = 1; break; }
      double alpha;
      if (it == 0) {
        if (!(del > 0.0)) { status = 2; break; }
        alpha = gam / del;
        for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
          const int i = beg + li;
          const double pi = ub[li], si = A.w[i];
          A.p[i] = pi;
          A.sv[i] = si;
          A.x[i] += alpha * pi;
          A.r[i] -= alpha * si;
        }
      } else {
        const double beta = gam / gam_prev;
        const double den = del - beta * gam / alpha_prev;
        if (!(den > 0.0) || !isfinite(den)) { status = 2; break; }
        alpha = gam / den;
        for (int li = threadIdx.x; li < nloc; li += blockDim.x) {
          const int i = beg + li;
          const double pi = ub[li] + beta * A.p[i];
          const double si = A.w[i] + beta * A.sv[i];
          A.p[i] = pi;
          A.sv[i] = si;
          A.x[i] += alpha * pi;
          A.r[i] -= alpha * si;
        }
      }
      gam_prev = gam;
      alpha_prev = alpha;
      cur ^= 1;
      ++it;
    }
  }
  // No CTA may leave while another can still read its shared memory.
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) {
    A.stat->iters = it;
    A.stat->status = status;
    A.stat->relres = bb > 0.0 ? sqrt(rho / bb) : 0.0;
    A.stat->bnorm = sqrt(bb);
  }
}

// ---------------------------------------------------------------------------
// Register-resident variant for unit-weight Laplacians with at most 6
// neighbours per row and at most VPT rows per thread: every per-row quantity
// (x, r, p, s, Jacobi and data diagonals, the 6 neighbour addresses) stays in
// registers for the whole solve, neighbours are read with one
// ld.shared::cluster each from addresses resolved once with mapa (a missing
// neighbour points at a zero word), and the iteration scalars are formed once
// per CTA by one thread.  Same Chronopoulos-Gear recurrence and reduction
// order as pcg_cluster_kernel.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t mapa_u32(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

template <class T>
__device__ __forceinline__ T ld_dsm(uint32_t a);

template <>
__device__ __forceinline__ double ld_dsm<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}

template <>
__device__ __forceinline__ float ld_dsm<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}

template <class T>
__device__ __forceinline__ T ld_sh(uint32_t a);

template <>
__device__ __forceinline__ double ld_sh<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}

template <>
__device__ __forceinline__ float ld_sh<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}

constexpr int kRegSlots = 6;

template <int KIND, int VPT, class T>
__global__ void __launch_bounds__(kPcgThreads, 1) pcg_reg_kernel(const PcgArgs A) {
  constexpr bool kF32 = sizeof(T) == sizeof(float);
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const DevLap& L = A.L;
  const int chunk = L.chunk;
  const int beg = rank * chunk;
  const int nloc = max(0, min(L.n - beg, chunk));
  const int m = A.m;
  extern __shared__ __align__(16) double sm[];
  // layout (doubles): [red 8] [ypart m] [sS m] [sY m] [scr 128] [scal 8]; then (T): [zero 2] [ub0] [ub1] [tb]
  double* red = sm;
  double* ypart = red + 8;
  double* sS = ypart + m;
  double* sY = sS + m;
  double* scr = sY + m;
  double* scal = scr + 128;
  T* zero = reinterpret_cast<T*>(scal + 8);
  T* ub0 = zero + 2;
  T* ub1 = ub0 + chunk;
  T* tb = ub1 + chunk;
  const uint32_t off_ub1 = (uint32_t)(chunk * sizeof(T));
  const uint32_t off_tb = (uint32_t)(2 * chunk * sizeof(T));
  const T lam = (T)A.lam;
  const double c = A.coef[0];
  const double d = A.coef[1];
  const T e = (T)(d - c * c);
  if (threadIdx.x == 0) {
    zero[0] = (T)0;
    zero[1] = (T)0;
  }
  for (int a = threadIdx.x; a < m; a += blockDim.x) sS[a] = KIND == 0 ? A.xi[a] * A.xi[a] : A.s[a];
  __syncthreads();

  T x[VPT], r[VPT], p[VPT], sv[VPT], dpc[VPT], dinv[VPT], omt[VPT];
  uint32_t na[VPT][kRegSlots];
  uint32_t rmask[VPT];  // bit q set: neighbour q lives in another CTA
  int xr0[VPT], xr1[VPT];
  bool own[VPT];
  const uint32_t zaddr = smem_u32(zero);
  const uint32_t base0 = smem_u32(ub0);
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int li = threadIdx.x + k * blockDim.x;
    own[k] = li < nloc;
    const int i = beg + (own[k] ? li : 0);
    x[k] = r[k] = p[k] = sv[k] = (T)0;
    dpc[k] = dinv[k] = omt[k] = (T)0;
    xr0[k] = xr1[k] = 0;
    rmask[k] = 0u;
#pragma unroll
    for (int q = 0; q < kRegSlots; ++q) na[k][q] = zaddr;
    if (own[k]) {
#pragma unroll
      for (int q = 0; q < kRegSlots; ++q) {
        if (q < L.K) {
          const int pk = L.nbrp[(size_t)q * L.n + i];
          // a missing neighbour reads the local zero word (no buffer offset is added to it)
          if (pk >= 0) {
            const uint32_t loc = base0 + (uint32_t)((pk & 0xFFFFFF) * sizeof(T));
            const int owner = pk >> 24;
            if (owner == rank) {
              na[k][q] = loc;
            } else {
              na[k][q] = mapa_u32(loc, (uint32_t)owner);
              rmask[k] |= 1u << q;
            }
          }
        }
      }
      dpc[k] = (T)(L.diag[i] + c);
      double dd = A.lam * (L.l2diag[i] + 2.0 * c * L.diag[i] + d);
      if (KIND == 0) {
        double o = 0.0;
        for (int a = 0; a < m; ++a) o += (double)A.Om[i + (int64_t)a * A.ldo] * sS[a];
        omt[k] = (T)o;
        dd += o;
      } else {
        xr0[k] = A.X.xr_ptr[i];
        xr1[k] = A.X.xr_ptr[i + 1];
        for (int q = xr0[k]; q < xr1[k]; ++q) dd += A.X.xr_val[q] * A.X.xr_val[q] * sS[A.X.xr_col[q]];
      }
      dinv[k] = (T)(dd > 0.0 ? 1.0 / dd : 1.0);
      x[k] = (T)A.x[i];
    }
  }

  // neighbour sum of the buffer at byte offset `off` from ub0 (zero word for a missing neighbour)
  // all six loads are issued before the first add (in-order issue would
  // otherwise serialise their latencies); the sum order is fixed
  auto nsum = [&](int k, uint32_t off) -> T {
    T v[kRegSlots];
#pragma unroll
    for (int q = 0; q < kRegSlots; ++q) {
      const uint32_t a = na[k][q];
      if ((rmask[k] >> q) & 1u)
        v[q] = ld_dsm<T>(a + off);
      else
        v[q] = ld_sh<T>(a == zaddr ? a : a + off);
    }
    return ((v[0] + v[1]) + (v[2] + v[3])) + (v[4] + v[5]);
  };
  // v side: partial X^T of the buffer in shared memory
  // (float32 kernel: the X data term runs in float32 on float32 copies of X;
  // ypart and sY then hold floats)
  float* ypart_f = reinterpret_cast<float*>(ypart);
  float* sY_f = reinterpret_cast<float*>(sY);
  float* sSf = ypart_f + m;  // float copy of sS in the upper half of the ypart words
  if (kF32)
    for (int a = threadIdx.x; a < m; a += blockDim.x) sSf[a] = (float)sS[a];
  auto ypartial = [&](T* buf) {
    if (KIND == 1) {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int a = wid; a < m; a += nw) {
        const int p0 = A.X.lx_ptr[rank * m + a], p1 = A.X.lx_ptr[rank * m + a + 1];
        if constexpr (kF32) {
          float acc = 0.f;
          for (int q = p0 + lane; q < p1; q += 32) acc += A.X.lx_valf[q] * buf[A.X.lx_row[q]];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
          if (lane == 0) ypart_f[a] = acc;
        } else {
          double acc = 0.0;
          for (int q = p0 + lane; q < p1; q += 32) acc += A.X.lx_val[q] * (double)buf[A.X.lx_row[q]];
          acc = warp_sum(acc);
          if (lane == 0) ypart[a] = acc;
        }
      }
    }
  };
  auto gather = [&]() {
    if (KIND == 1) {
      for (int a = threadIdx.x; a < m; a += blockDim.x) {
        if constexpr (kF32) {
          float pv[kMaxCluster];
#pragma unroll
          for (int rr = 0; rr < kMaxCluster; ++rr)
            pv[rr] = rr < C ? cl.map_shared_rank(ypart_f, (unsigned)rr)[a] : 0.f;
          float t = 0.f;
#pragma unroll
          for (int rr = 0; rr < kMaxCluster; ++rr) t += pv[rr];
          sY_f[a] = sSf[a] * t;
        } else {
          double pv[kMaxCluster];
#pragma unroll
          for (int rr = 0; rr < kMaxCluster; ++rr) pv[rr] = rr < C ? cl.map_shared_rank(ypart, (unsigned)rr)[a] : 0.0;
          double t = 0.0;
#pragma unroll
          for (int rr = 0; rr < kMaxCluster; ++rr) t += pv[rr];
          sY[a] = sS[a] * t;
        }
      }
      __syncthreads();
    }
  };
  auto data = [&](int k, T ui) -> T {
    if (KIND == 0) return omt[k] * ui;
    if constexpr (kF32) {
      float acc = 0.f;
      for (int q = xr0[k]; q < xr1[k]; ++q) acc += A.X.xr_valf[q] * sY_f[A.X.xr_col[q]];
      return acc;
    } else {
      double acc = 0.0;
      for (int q = xr0[k]; q < xr1[k]; ++q) acc += A.X.xr_val[q] * sY[A.X.xr_col[q]];
      return (T)acc;
    }
  };

  // r0 = b - A x0
  T tt[VPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k)
    if (own[k]) ub0[threadIdx.x + k * blockDim.x] = x[k];
  cl.sync();
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    tt[k] = own[k] ? dpc[k] * x[k] - nsum(k, 0) : (T)0;
    if (own[k]) tb[threadIdx.x + k * blockDim.x] = tt[k];
  }
  ypartial(ub0);
  cl.sync();
  gather();
  double bb;
  if constexpr (kF32) {
    DF v1[1] = {DF{0.f, 0.f}};
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (!own[k]) continue;
      const int i = beg + threadIdx.x + k * blockDim.x;
      const T wi = lam * (dpc[k] * tt[k] - nsum(k, off_tb) + e * x[k]) + data(k, x[k]);
      const float bi = (float)A.b[i];
      r[k] = bi - wi;
      v1[0] = df_add(v1[0], df_prod(bi, bi));
    }
    block_sum_df<1>(v1, reinterpret_cast<DF*>(scr), reinterpret_cast<DF*>(red));
    cl.sync();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      DF g{0.f, 0.f};
      if (lane < C) g = cl.map_shared_rank(reinterpret_cast<DF*>(red), lane)[0];
      g = warp_sum_df(g);
      if (lane == 0) reinterpret_cast<DF*>(scal)[0] = g;
    }
    __syncthreads();
    const DF b2 = reinterpret_cast<const DF*>(scal)[0];
    bb = (double)b2.hi + (double)b2.lo;
  } else {
    double v[1] = {0.0};
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      if (!own[k]) continue;
      const int i = beg + threadIdx.x + k * blockDim.x;
      const T wi = lam * (dpc[k] * tt[k] - nsum(k, off_tb) + e * x[k]) + data(k, x[k]);
      const double bi = A.b[i];
      r[k] = (T)(bi - (double)wi);
      v[0] += bi * bi;
    }
    block_sum<1>(v, scr, red);
    cl.sync();
    cluster_sum<1>(cl, red, scal, C);
    bb = scal[0];
  }
  int it = 0, status = 0;
  double rho = 0.0;
  DF rho_df{0.f, 0.f};
  if (bb > 0.0) {
    const double tol2 = A.tol * A.tol * bb;
    const float tol2f = (float)tol2;
    double gam_prev = 1.0, alpha_prev = 1.0;  // used by thread 0 only
    DF gam_prev_df{1.f, 0.f}, alpha_prev_df{1.f, 0.f};
    int cur = 1;
    for (;;) {
      const uint32_t off_ub = cur ? off_ub1 : 0u;
      T* ub = cur ? ub1 : ub0;
      T u[VPT];
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        u[k] = r[k] * dinv[k];
        if (own[k]) ub[threadIdx.x + k * blockDim.x] = u[k];
      }
      cl.sync();
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        tt[k] = own[k] ? dpc[k] * u[k] - nsum(k, off_ub) : (T)0;
        if (own[k]) tb[threadIdx.x + k * blockDim.x] = tt[k];
      }
      ypartial(ub);
      cl.sync();
      gather();
      T w[VPT];
#pragma unroll
      for (int k = 0; k < VPT; ++k)
        w[k] = own[k] ? lam * (dpc[k] * tt[k] - nsum(k, off_tb) + e * u[k]) + data(k, u[k]) : (T)0;
      if constexpr (kF32) {
        // inner products from exact float products, summed in double-float
        DF v3[3] = {DF{0.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}};
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          v3[0] = df_add(v3[0], df_prod(r[k], u[k]));
          v3[1] = df_add(v3[1], df_prod(u[k], w[k]));
          v3[2] = df_add(v3[2], df_prod(r[k], r[k]));
        }
        block_sum_df<3>(v3, reinterpret_cast<DF*>(scr), reinterpret_cast<DF*>(red));
        cl.sync();
        if (threadIdx.x < 32) {
          const int lane = threadIdx.x;
          DF g{0.f, 0.f}, dl{0.f, 0.f}, rh{0.f, 0.f};
          if (lane < C) {
            const DF* rr = cl.map_shared_rank(reinterpret_cast<DF*>(red), lane);
            g = rr[0];
            dl = rr[1];
            rh = rr[2];
          }
          g = warp_sum_df(g);
          dl = warp_sum_df(dl);
          rh = warp_sum_df(rh);
          if (lane == 0) {
            float flag = 0.f;
            DF alpha{0.f, 0.f}, beta{0.f, 0.f};
            if (rh.hi <= tol2f) {
              flag = 1.f;
            } else if (it >= A.maxit) {
              flag = 2.f;
            } else {
              DF den = dl;
              if (it > 0) {
                beta = df_div(g, gam_prev_df);
                den = df_sub(dl, df_div(df_mul(beta, g), alpha_prev_df));
              }
              if (!(den.hi > 0.f) || !isfinite(den.hi)) {
                flag = 3.f;
              } else {
                alpha = df_div(g, den);
                gam_prev_df = g;
                alpha_prev_df = alpha;
              }
            }
            float* sf = reinterpret_cast<float*>(scal);
            sf[0] = flag;
            sf[1] = alpha.hi;
            sf[2] = beta.hi;
            sf[3] = rh.hi;
            sf[4] = rh.lo;
          }
        }
        __syncthreads();
      } else {
      double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        v[0] += (double)(r[k] * u[k]);
        v[1] += (double)(u[k] * w[k]);
        v[2] += (double)(r[k] * r[k]);
      }
      block_sum<3>(v, scr, red);
      cl.sync();
      // cross-CTA sums and the recurrence scalars, formed once per CTA
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double g = 0.0, dl = 0.0, rh = 0.0;
        if (lane < C) {
          const double* rr = cl.map_shared_rank(red, lane);
          g = rr[0];
          dl = rr[1];
          rh = rr[2];
        }
        g = warp_sum(g);
        dl = warp_sum(dl);
        rh = warp_sum(rh);
        if (lane == 0) {
          // gam_prev / alpha_prev hold 1/gamma_{i-1} and 1/alpha_{i-1}: one
          // division on the dependent chain (1/gamma_i is formed alongside)
          double flag = 0.0, alpha = 0.0, beta = 0.0;
          if (rh <= tol2) {
            flag = 1.0;
          } else if (it >= A.maxit) {
            flag = 2.0;
          } else {
            double den = dl;
            if (it > 0) {
              beta = g * gam_prev;
              den = dl - beta * g * alpha_prev;
            }
            if (!(den > 0.0) || !isfinite(den)) {
              flag = 3.0;
            } else {
              alpha = g / den;
              gam_prev = 1.0 / g;
              alpha_prev = den * gam_prev;
            }
          }
          scal[0] = flag;
          scal[1] = alpha;
          scal[2] = beta;
          scal[3] = rh;
        }
      }
      __syncthreads();
      }
      double flag;
      T alpha, beta;
      if constexpr (kF32) {
        const float* sf = reinterpret_cast<const float*>(scal);
        flag = sf[0];
        alpha = sf[1];
        beta = sf[2];
        rho_df = DF{sf[3], sf[4]};
      } else {
        flag = scal[0];
        rho = scal[3];
        alpha = (T)scal[1];
        beta = (T)scal[2];
      }
      if (flag == 1.0) break;
      if (flag == 2.0) {
        status = 1;
        break;
      }
      if (flag == 3.0) {
        status = 2;
        break;
      }
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        p[k] = it == 0 ? u[k] : u[k] + beta * p[k];
        sv[k] = it == 0 ? w[k] : w[k] + beta * sv[k];
        x[k] += alpha * p[k];
        r[k] -= alpha * sv[k];
      }
      cur ^= 1;
      ++it;
    }
  }
#pragma unroll
  for (int k = 0; k < VPT; ++k)
    if (own[k]) A.x[beg + threadIdx.x + k * blockDim.x] = (double)x[k];
  cl.sync();  // no CTA leaves while another can still read its shared memory
  if (rank == 0 && threadIdx.x == 0) {
    if constexpr (kF32) rho = (double)rho_df.hi + (double)rho_df.lo;
    A.stat->iters = it;
    A.stat->status = status;
    A.stat->relres = bb > 0.0 ? sqrt(rho / bb) : 0.0;
    A.stat->bnorm = sqrt(bb);
  }
}

__global__ void lap_apply_kernel(const DevLap L, const double* __restrict__ x, double* __restrict__ y,
                                 double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  double acc = (L.diag[i] + shift) * x[i];
  for (int k = 0; k < L.K; ++k) {
    const int q = L.nbr[(size_t)k * L.n + i];
    if (q < 0) continue;
    acc += (L.offw ? L.offw[(size_t)k * L.n + i] : -1.0) * x[q];
  }
  y[i] = acc;
}

}  // namespace

size_t pcg_smem_bytes(int chunk, int m) { return sizeof(double) * (3 * (size_t)chunk + 8 + 3 * (size_t)m + 128 + 8 + 2); }

// Register-resident variant usable for this operator?  Returns VPT (0 = no).
int pcg_reg_vpt(const DevLap& L, bool fp32) {
  if (L.offw != nullptr || L.K > kRegSlots) return 0;
  if (L.chunk <= kPcgThreads) return 1;
  if (L.chunk <= 2 * kPcgThreads) return 2;
  if (fp32 && L.chunk <= 4 * kPcgThreads) return 4;
  return 0;
}

cudaError_t pcg_prepare(int /*data_kind*/, int csize, size_t /*smem_bytes*/) {
  // the attribute is per kernel, shared by the x and y grids: allow the maximum
  const size_t smem_bytes = 227 * 1024;
  cudaError_t e;
  const void* fns[14] = {(const void*)pcg_cluster_kernel<0>,         (const void*)pcg_cluster_kernel<1>,
                         (const void*)pcg_reg_kernel<0, 1, double>, (const void*)pcg_reg_kernel<1, 1, double>,
                         (const void*)pcg_reg_kernel<0, 2, double>, (const void*)pcg_reg_kernel<1, 2, double>,
                         (const void*)pcg_reg_kernel<0, 1, float>,  (const void*)pcg_reg_kernel<1, 1, float>,
                         (const void*)pcg_reg_kernel<0, 2, float>,  (const void*)pcg_reg_kernel<1, 2, float>,
                         (const void*)pcg_reg_kernel<0, 4, float>,  (const void*)pcg_reg_kernel<1, 4, float>,
                         (const void*)pcg_reg_kernel<0, 4, float>,  (const void*)pcg_reg_kernel<1, 4, float>};
  for (int kind = 0; kind < 14; ++kind) {
    const void* fn = fns[kind];
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

bool pcg_cluster_ok(int cs, size_t smem_bytes) {
  if (pcg_prepare(0, cs, smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = smem_bytes;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  for (int kind = 0; kind < 2; ++kind) {
    const void* fn = kind == 0 ? (const void*)pcg_cluster_kernel<0> : (const void*)pcg_cluster_kernel<1>;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return false;
    }
  }
  return true;
}

cudaError_t pcg_launch(const PcgArgs& a, int data_kind, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.L.csize);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = pcg_smem_bytes(a.L.chunk, a.m);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = a.L.csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  const bool f32 = a.fp32 != 0;
  const int vpt = a.force_generic ? 0 : pcg_reg_vpt(a.L, f32);
  if (f32) {
    if (vpt == 1) return data_kind == 0 ? cudaLaunchKernelEx(&cfg, pcg_reg_kernel<0, 1, float>, a)
                                        : cudaLaunchKernelEx(&cfg, pcg_reg_kernel<1, 1, float>, a);
    if (vpt == 2) return data_kind == 0 ? cudaLaunchKernelEx(&cfg, pcg_reg_kernel<0, 2, float>, a)
                                        : cudaLaunchKernelEx(&cfg, pcg_reg_kernel<1, 2, float>, a);
    if (vpt == 4) return data_kind == 0 ? cudaLaunchKernelEx(&cfg, pcg_reg_kernel<0, 4, float>, a)
                                        : cudaLaunchKernelEx(&cfg, pcg_reg_kernel<1, 4, float>, a);
  }
  if (vpt == 1) {
    if (data_kind == 0) return cudaLaunchKernelEx(&cfg, pcg_reg_kernel<0, 1, double>, a);
    return cudaLaunchKernelEx(&cfg, pcg_reg_kernel<1, 1, double>, a);
  }
  if (vpt == 2) {
    if (data_kind == 0) return cudaLaunchKernelEx(&cfg, pcg_reg_kernel<0, 2, double>, a);
    return cudaLaunchKernelEx(&cfg, pcg_reg_kernel<1, 2, double>, a);
  }
  if (data_kind == 0) return cudaLaunchKernelEx(&cfg, pcg_cluster_kernel<0>, a);
  return cudaLaunchKernelEx(&cfg, pcg_cluster_kernel<1>, a);
}

void lap_apply(const DevLap& L, const double* x, double* y, double shift, cudaStream_t st) {
  if (L.n == 0) return;
  count_launch();
  lap_apply_kernel<<<(L.n + 255) / 256, 256, 0, st>>>(L, x, y, shift);
}

}  // namespace cr
