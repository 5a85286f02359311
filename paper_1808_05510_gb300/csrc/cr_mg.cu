// Multigrid-preconditioned CG for the ALS sub-problems (Sec. 2.3, Eqs.
// ALS_linsys and ALS_linsys_v), one thread-block cluster per solve.
//
// The operators are  lam [(L + cI)^2 + e I] + data  (see cr_pcg.cu).  The paper
// solves these systems directly; as matrix-free PCG they are badly conditioned
// (hundreds to thousands of Jacobi-PCG iterations for the smooth ALS factors).
// The preconditioner here is
//     M^-1 r = (1 / lam) V(V(r)),
// V one V-cycle for the shifted Laplacian L + sigma I, with
//     sigma^2 = c^2 + e + wbar / lam = d + wbar / lam,
// wbar the mean data weight: u side sum_a xi_a^2 (the weight of a voxel that
// is observed in every injection), v side sum_a s_a |X_a|^2 / n.  Then
// lam (L + sigma I)^2 matches the operator's Laplacian part up to a factor in
// [1/2, 1] on every eigenvector of L, and two V-cycles approximate its inverse.
// V is symmetric (pre- and post-smoothing mirror each other, restriction is
// the transpose of prolongation), so V(V(.)) is symmetric positive definite
// and plain (Chronopoulos-Gear) PCG applies.
//
// V-cycle: on every level two damped-Jacobi sweeps (omega = 2/3) before and
// after the coarse correction; the coarsest level (at most kMgCoarseMax rows)
// is solved exactly through the eigenbasis of the pencil (L_c, M_c) computed
// once on the host, so no factorisation happens per shift.
//
// Layout: level 0 is the fine grid, in the cluster's chunk partition (the
// neighbour table of DevLap); levels with more than kMgTailRows rows are
// partitioned over the cluster too; the smaller levels and the coarsest run on
// CTA 0 alone with CTA-local barriers.  Every level keeps its vectors in
// shared memory; neighbours in other CTAs are read through distributed shared
// memory.  Reductions use a fixed order (warps, then CTAs in rank order), so
// every CTA forms identical scalars and takes the same branches, and results
// repeat run to run.  Cluster barriers per PCG iteration: 3 for the operator
// and the inner products, 5 + 6 (distributed levels - 1) + 1 per V-cycle.
// Rows of the coarse levels hold tens of entries (smoothed aggregation), so a
// group of lanes shares each row and sums by shuffles: the loads of a row are
// in flight together instead of one dependent load after another.
#include <cooperative_groups.h>

#include "cr_common.cuh"

namespace cg = cooperative_groups;

namespace cr {

namespace {

constexpr double kOmega = 2.0 / 3.0;

__device__ __forceinline__ double mg_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NV>
__device__ __forceinline__ void mg_block_sum(double (&v)[NV], double* scr, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = mg_warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) scr[wid * NV + q] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = lane < nw ? scr[lane * NV + q] : 0.0;
      t = mg_warp_sum(t);
      if (lane == 0) out[q] = t;
    }
  }
}

// After a cluster barrier: the NV partial sums of all CTAs in rank order, into scal[].
template <int NV>
__device__ __forceinline__ void mg_cluster_sum(cg::cluster_group& cl, double* red, double* scal, int csize) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      if (lane < csize) t = cl.map_shared_rank(red, lane)[q];
      t = mg_warp_sum(t);
      if (lane == 0) scal[q] = t;
    }
  }
  __syncthreads();
}

template <class T>
__device__ __forceinline__ T ld_ref(cg::cluster_group& cl, T* buf, int ref) {
  return cl.map_shared_rank(buf, (unsigned)(ref >> 24))[ref & 0xFFFFFF];
}

// Sum over the G lanes of each aligned lane group (G a power of two <= 32); lane 0 of the group gets it.
template <class T>
__device__ __forceinline__ T group_sum(T v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, G);
  return v;
}

template <int KIND, class T>
__global__ void __launch_bounds__(kPcgThreads, 1) pcg_mg_kernel(const PcgArgs A, const DevMg G) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, nth = blockDim.x;
  const DevLap& L = A.L;
  const int chunk0 = L.chunk;
  const int beg0 = rank * chunk0;
  const int n0 = max(0, min(L.n - beg0, chunk0));
  const int m = A.m;
  const int nc = G.nc;
  extern __shared__ __align__(16) double sm[];
  double* red = sm;             // [8]
  double* scr = red + 8;        // [128]
  double* scal = scr + 128;     // [16]
  double* ypart = scal + 16;    // [m]
  double* sS = ypart + m;       // [m]  xi^2 (u side) or s (v side)
  double* sY = sS + m;          // [m]  s (X^T u) (v side)
  double* cQ = sY + m;          // [nc * nc]
  double* cmu = cQ + nc * nc;   // [nc]
  double* ctmp = cmu + nc;      // [nc]
  T* u = reinterpret_cast<T*>(ctmp + nc);
  T* t = u + chunk0;
  T* r = t + chunk0;
  T* wv = r + chunk0;
  T* y = wv + chunk0;
  T* xa0 = y + chunk0;
  T* xb0 = xa0 + chunk0;
  T* di0 = xb0 + chunk0;    // 1 / diag(L + sigma I), own rows
  T* lvl = di0 + chunk0;    // levels >= 1: [xa | xb | rr | tt | dinv] of `chunk` elements each, at G.lev[l].off

  const double lam = A.lam;
  const double c = A.coef[0];
  const double d = A.coef[1];
  const double e = d - c * c;

  for (int a = tid; a < m; a += nth) sS[a] = KIND == 0 ? A.xi[a] * A.xi[a] : A.s[a];
  if (rank == 0)
    for (int q = tid; q < nc * nc; q += nth) cQ[q] = G.cQ[q];
  if (rank == 0)
    for (int q = tid; q < nc; q += nth) cmu[q] = G.cmu[q];
  __syncthreads();
  // shift of the V-cycles (identical in every thread: fixed summation order)
  double wbar = 0.0;
  if (KIND == 0) {
    for (int a = 0; a < m; ++a) wbar += sS[a];
  } else {
    for (int a = 0; a < m; ++a) wbar += sS[a] * G.xn2[a];
    wbar /= (double)L.n;
  }
  const double sig2 = fmax(d + wbar / lam, 1e-12);
  const double sigd = sqrt(sig2);
  const T sig = (T)sigd;
  const T om = (T)kOmega;

  // ---- level helpers -------------------------------------------------------------
  auto nown = [&](int l) -> int {
    const DevMgLevel& V = G.lev[l];
    if (!V.dist) return rank == 0 ? V.n : 0;
    return max(0, min(V.n - rank * V.chunk, V.chunk));
  };
  auto gbeg = [&](int l) -> int { return l == 0 ? beg0 : (G.lev[l].dist ? rank * G.lev[l].chunk : 0); };
  auto bufs = [&](int l, int k) -> T* {  // k: 0 xa, 1 xb, 2 rr, 3 tt, 4 dinv
    if (l == 0) return k == 0 ? xa0 : k == 1 ? xb0 : k == 3 ? t : di0;
    return lvl + G.lev[l].off + k * G.lev[l].chunk;
  };
  // lanes per row for a level with `rows` rows in this CTA: rows times lanes fill the CTA
  auto gsize = [&](int rows) -> int {
    int g = 1;
    while (g < 32 && 2 * g * rows <= nth) g *= 2;
    return g;
  };

  // per-row set-up: data diagonal (u side) and the inverse Jacobi diagonals of every level
  if (KIND == 0) {
    for (int li = tid; li < n0; li += nth) {
      const int i = beg0 + li;
      double o = 0.0;
      for (int a = 0; a < m; ++a) o += (double)A.Om[i + (int64_t)a * A.ldo] * sS[a];
      A.omt[i] = o;
    }
  }
  for (int li = tid; li < n0; li += nth) di0[li] = (T)(1.0 / (L.diag[beg0 + li] + sigd));
  for (int l = 1; l < G.nlev - 1; ++l) {  // the coarsest level is solved through its eigenbasis: no diagonal
    const int no = nown(l), gb = gbeg(l);
    T* dv = bufs(l, 4);
    for (int li = tid; li < no; li += nth) {
      const double dd = G.lev[l].dl[gb + li] + sigd * G.lev[l].dm[gb + li];
      dv[li] = (T)(dd > 0.0 ? 1.0 / dd : 0.0);
    }
  }

  // (L + shift I) x on level 0, row li of this CTA, x in the cluster-partitioned buffer `buf`;
  // up to six neighbours: every reference and value load is issued before the first add
  auto lap0 = [&](int li, T* buf, T shift) -> T {
    const int i = beg0 + li;
    T acc = ((T)L.diag[i] + shift) * buf[li];
    if (L.K <= 6) {
      int q[6];
      T nv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) q[k] = k < L.K ? __ldg(L.nbrp + (size_t)k * L.n + i) : -1;
#pragma unroll
      for (int k = 0; k < 6; ++k) nv[k] = q[k] >= 0 ? ld_ref(cl, buf, q[k]) : (T)0;
      if (L.offw) {
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (q[k] >= 0) acc += (T)__ldg(L.offw + (size_t)k * L.n + i) * nv[k];
      } else {
        acc -= ((nv[0] + nv[1]) + (nv[2] + nv[3])) + (nv[4] + nv[5]);
      }
      return acc;
    }
    for (int k = 0; k < L.K; ++k) {
      const int q = __ldg(L.nbrp + (size_t)k * L.n + i);
      if (q < 0) continue;
      acc += (L.offw ? (T)__ldg(L.offw + (size_t)k * L.n + i) : (T)-1) * ld_ref(cl, buf, q);
    }
    return acc;
  };
  // this lane's share of ((L_l + sigma M_l) x)_gi, entries lane, lane + G, ... of the row
  auto lapl_part = [&](int l, int gi, int lane, int g, T* buf) -> T {
    const DevMgLevel& V = G.lev[l];
    T acc = (T)0;
    const int q1 = V.rp[gi + 1];
    for (int q = V.rp[gi] + lane; q < q1; q += g) acc += ((T)V.lv[q] + sig * (T)V.mv[q]) * ld_ref(cl, buf, V.cp[q]);
    return acc;
  };
  // Row sweep on level l with one lane group per row: part(li, lane, g) returns a
  // lane's partial sum (level 0: one lane per row, the whole row), fin(li, sum)
  // stores the row's result.  The loop bounds are uniform over the CTA, so every
  // lane of every warp takes part in the group shuffles.
  auto sweep = [&](int l, auto&& part, auto&& fin) {
    const int no = nown(l);
    if (l == 0) {
      for (int li = tid; li < no; li += nth) fin(li, part(li, 0, 1));
      return;
    }
    const int g = gsize(no), rpp = nth / g, lane = tid % g;
    for (int base = 0; base < no; base += rpp) {
      const int li = base + tid / g;
      T s = li < no ? part(li, lane, g) : (T)0;
      s = group_sum(s, g);
      if (li < no && lane == 0) fin(li, s);
    }
  };
  // (A_l x) row share on level l
  auto arow = [&](int l, T* buf) {
    return [&, l, buf](int li, int lane, int g) -> T {
      if (l == 0) return lap0(li, buf, sig);
      return lapl_part(l, gbeg(l) + li, lane, g, buf);
    };
  };
  // level barriers: cluster-wide on distributed levels, CTA-local on CTA 0's levels
  auto lsync = [&](int l) {
    if (G.lev[l].dist)
      cl.sync();
    else
      __syncthreads();
  };
  // pre-smoothing and residual on level l (rhs R), then restriction into level l+1
  auto down = [&](int l, T* R) {
    T* xa = bufs(l, 0);
    T* xb = bufs(l, 1);
    T* tt = bufs(l, 3);
    T* dv = bufs(l, 4);
    const int no = nown(l);
    for (int li = tid; li < no; li += nth) xa[li] = om * R[li] * dv[li];
    lsync(l);
    sweep(l, arow(l, xa), [&](int li, T ax) { xb[li] = xa[li] + om * (R[li] - ax) * dv[li]; });
    lsync(l);
    sweep(l, arow(l, xb), [&](int li, T ax) { tt[li] = R[li] - ax; });
    lsync(l);
    // restriction: rows of level l+1 owned here (CTA 0 owns all rows of its levels)
    const DevMgLevel& V = G.lev[l];
    T* rn = bufs(l + 1, 2);
    const int gbn = gbeg(l + 1);
    sweep(
        l + 1,
        [&](int lj, int lane, int g) -> T {
          const int gj = gbn + lj;
          T acc = (T)0;
          const int q1 = V.rrp[gj + 1];
          for (int q = V.rrp[gj] + lane; q < q1; q += g) acc += (T)V.rv[q] * ld_ref(cl, tt, V.rcp[q]);
          return acc;
        },
        [&](int lj, T v) { rn[lj] = v; });
    // lane 0 of a group wrote each row; the next level's first sweep reads it one thread per row
    __syncthreads();
  };
  // coarse correction from level l+1, post-smoothing on level l; result in OUT (times scale)
  auto up = [&](int l, T* R, T* OUT, T scale) {
    T* xa = bufs(l, 0);
    T* xb = bufs(l, 1);
    T* dv = bufs(l, 4);
    const DevMgLevel& V = G.lev[l];
    T* xc = bufs(l + 1, 0);
    const int gb = gbeg(l);
    sweep(
        l,
        [&](int li, int lane, int g) -> T {
          const int gi = gb + li;
          T acc = (T)0;
          const int q1 = V.prp[gi + 1];
          for (int q = V.prp[gi] + lane; q < q1; q += g) acc += (T)V.pv[q] * ld_ref(cl, xc, V.pcp[q]);
          return acc;
        },
        [&](int li, T v) { xa[li] = xb[li] + v; });
    lsync(l);
    sweep(l, arow(l, xa), [&](int li, T ax) { xb[li] = xa[li] + om * (R[li] - ax) * dv[li]; });
    lsync(l);
    sweep(l, arow(l, xb), [&](int li, T ax) { OUT[li] = scale * (xb[li] + om * (R[li] - ax) * dv[li]); });
  };
  // exact solve on the coarsest level (CTA 0): x = Q diag(1 / (mu + sigma)) Q^T r
  auto coarse = [&]() {
    __syncthreads();  // the restriction into the coarsest level wrote rows of other threads
    T* rc = bufs(G.nlev - 1, 2);
    T* xc = bufs(G.nlev - 1, 0);
    for (int k = tid; k < nc; k += nth) {
      double acc = 0.0;
      for (int i = 0; i < nc; ++i) acc += cQ[i + k * nc] * (double)rc[i];
      ctmp[k] = acc / (fmax(cmu[k], 0.0) + sigd);
    }
    __syncthreads();
    for (int i = tid; i < nc; i += nth) {
      double acc = 0.0;
      for (int k = 0; k < nc; ++k) acc += cQ[i + k * nc] * ctmp[k];
      xc[i] = (T)acc;
    }
    __syncthreads();
  };
  // one V-cycle: OUT = scale * V(R) on level 0 (own rows)
  auto vcycle = [&](T* R, T* OUT, T scale) {
    const int ld = G.ld;
    for (int l = 0; l < ld; ++l) down(l, l == 0 ? R : bufs(l, 2));
    if (rank == 0) {
      for (int l = ld; l < G.nlev - 1; ++l) down(l, bufs(l, 2));
      coarse();
      for (int l = G.nlev - 2; l >= ld; --l) {
        up(l, bufs(l, 2), bufs(l, 0), (T)1);
        __syncthreads();
      }
    }
    cl.sync();
    for (int l = ld - 1; l >= 0; --l) {
      if (l == 0) {
        up(0, R, OUT, scale);
      } else {
        up(l, bufs(l, 2), bufs(l, 0), (T)1);
        lsync(l);
      }
    }
  };

  // ---- PCG (Chronopoulos-Gear) ------------------------------------------------------
  // operator: t = (L + cI) z; w = lam ((L + cI) t + e z) + data(z); v side: partial X^T z
  auto ypartial = [&](T* z) {
    if (KIND == 1) {
      const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
      for (int a = wid; a < m; a += nw) {
        const int p0 = A.X.lx_ptr[rank * m + a], p1 = A.X.lx_ptr[rank * m + a + 1];
        double acc = 0.0;
        for (int q = p0 + lane; q < p1; q += 32) acc += A.X.lx_val[q] * (double)z[A.X.lx_row[q]];
        acc = mg_warp_sum(acc);
        if (lane == 0) ypart[a] = acc;
      }
    }
  };
  auto gather = [&]() {
    if (KIND == 1) {
      for (int a = tid; a < m; a += nth) {
        double s = 0.0;
        for (int q = 0; q < C; ++q) s += cl.map_shared_rank(ypart, (unsigned)q)[a];
        sY[a] = sS[a] * s;
      }
      __syncthreads();
    }
  };
  auto data = [&](int li, T zi) -> T {
    const int i = beg0 + li;
    if (KIND == 0) return (T)A.omt[i] * zi;
    double acc = 0.0;
    for (int q = A.X.xr_ptr[i]; q < A.X.xr_ptr[i + 1]; ++q) acc += A.X.xr_val[q] * sY[A.X.xr_col[q]];
    return (T)acc;
  };
  const T cT = (T)c, lamT = (T)lam, eT = (T)e;

  // r0 = b - A x0
  for (int li = tid; li < n0; li += nth) u[li] = (T)A.x[beg0 + li];
  cl.sync();
  for (int li = tid; li < n0; li += nth) t[li] = lap0(li, u, cT);
  ypartial(u);
  cl.sync();
  gather();
  {
    double v1[1] = {0.0};
    for (int li = tid; li < n0; li += nth) {
      const int i = beg0 + li;
      const T wi = lamT * (lap0(li, t, cT) + eT * u[li]) + data(li, u[li]);
      const double bi = A.b[i];
      r[li] = (T)(bi - (double)wi);
      v1[0] += bi * bi;
    }
    mg_block_sum<1>(v1, scr, red);
  }
  cl.sync();
  mg_cluster_sum<1>(cl, red, scal, C);
  const double bb = scal[0];
  int it = 0, status = 0;
  double rho = 0.0;
  if (bb > 0.0) {
    const double tol2 = A.tol * A.tol * bb;
    double gam_prev = 1.0, alpha_prev = 1.0;
    for (;;) {
      // u = M^-1 r = (1 / lam) V(V(r))
      vcycle(r, y, (T)1);
      vcycle(y, u, (T)(1.0 / lam));
      cl.sync();
      for (int li = tid; li < n0; li += nth) t[li] = lap0(li, u, cT);
      ypartial(u);
      cl.sync();
      gather();
      double v[3] = {0.0, 0.0, 0.0};
      for (int li = tid; li < n0; li += nth) {
        const T ui = u[li];
        const T wi = lamT * (lap0(li, t, cT) + eT * ui) + data(li, ui);
        const T ri = r[li];
        wv[li] = wi;
        v[0] += (double)ri * (double)ui;
        v[1] += (double)ui * (double)wi;
        v[2] += (double)ri * (double)ri;
      }
      mg_block_sum<3>(v, scr, red);
      cl.sync();
      mg_cluster_sum<3>(cl, red, scal, C);
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
      const T aT = (T)alpha, bT = (T)beta;
      for (int li = tid; li < n0; li += nth) {
        const int i = beg0 + li;
        const T pi = it == 0 ? u[li] : u[li] + bT * (T)A.p[i];
        const T si = it == 0 ? wv[li] : wv[li] + bT * (T)A.sv[i];
        A.p[i] = (double)pi;
        A.sv[i] = (double)si;
        A.x[i] = (double)((T)A.x[i] + aT * pi);
        r[li] = r[li] - aT * si;
      }
      gam_prev = gam;
      alpha_prev = alpha;
      ++it;
    }
  } else {
    for (int li = tid; li < n0; li += nth) A.x[beg0 + li] = 0.0;
  }
  cl.sync();  // no CTA leaves while another can still read its shared memory
  if (rank == 0 && tid == 0) {
    A.stat->iters = it;
    A.stat->status = status;
    A.stat->relres = bb > 0.0 ? sqrt(rho / bb) : 0.0;
    A.stat->bnorm = sqrt(bb);
  }
}

}  // namespace

size_t mg_smem_bytes(const DevMg& g, int chunk0, int m, bool fp32) {
  const size_t tsz = fp32 ? sizeof(float) : sizeof(double);
  const size_t dbl = 8 + 128 + 16 + 3 * (size_t)m + (size_t)g.nc * g.nc + 2 * (size_t)g.nc;
  return sizeof(double) * dbl + tsz * (8 * (size_t)chunk0 + (size_t)g.lvl_elems) + 16;
}

cudaError_t mg_prepare() {
  const void* fns[4] = {(const void*)pcg_mg_kernel<0, double>, (const void*)pcg_mg_kernel<1, double>,
                        (const void*)pcg_mg_kernel<0, float>, (const void*)pcg_mg_kernel<1, float>};
  for (const void* fn : fns) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool mg_cluster_ok(int csize, size_t smem, bool fp32) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  const void* fn = fp32 ? (const void*)pcg_mg_kernel<1, float> : (const void*)pcg_mg_kernel<1, double>;
  if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess || ncl < 1) {
    cudaGetLastError();
    return false;
  }
  return true;
}

cudaError_t mg_pcg_launch(const PcgArgs& a, const DevMg& g, int side, cudaStream_t st) {
  const bool f32 = a.fp32 != 0;
  const size_t smem = g.smem[f32 ? 0 : 1];
  if (g.nlev < 2 || smem == 0 || a.L.csize < 1) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.L.csize);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = a.L.csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  if (f32) {
    if (side == 0) return cudaLaunchKernelEx(&cfg, pcg_mg_kernel<0, float>, a, g);
    return cudaLaunchKernelEx(&cfg, pcg_mg_kernel<1, float>, a, g);
  }
  if (side == 0) return cudaLaunchKernelEx(&cfg, pcg_mg_kernel<0, double>, a, g);
  return cudaLaunchKernelEx(&cfg, pcg_mg_kernel<1, double>, a, g);
}

}  // namespace cr
