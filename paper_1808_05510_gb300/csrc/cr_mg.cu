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
// in flight together instead of one dependent load after another.  At launch
// every CTA resolves, for the rows it owns, each referenced entry to its 32-bit
// cluster-window address (mapa) and its coefficient in the solve's precision
// (L_l + sigma M_l for the shift of this solve); the sweeps then read
// neighbours with one ld.shared::cluster each.
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

__device__ __forceinline__ uint32_t mg_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t mg_mapa(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

template <class T>
__device__ __forceinline__ T mg_ld(uint32_t a);
// Volatile (never merged or dropped, kept in order among themselves and with the
// barriers, which are volatile too) but without a memory clobber, so that the
// loads of a row are issued back to back before their values are used.
template <>
__device__ __forceinline__ double mg_ld<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
template <>
__device__ __forceinline__ float mg_ld<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
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
  // v side with the Sherman-Morrison-Woodbury correction: [m*m] partial X^T MX, [m*m] X^T MX,
  // [m*m] (I + D X^T MX D)^-1, [m] D X^T y, [m] the correction's coefficients
  const bool smw = KIND == 1 && G.smw;
  double* smw_part = ctmp + nc;
  double* smw_xx = smw_part + (smw ? m * m : 0);
  double* smw_ci = smw_xx + (smw ? m * m : 0);
  double* smw_xt = smw_ci + (smw ? m * m : 0);
  double* smw_g = smw_xt + (smw ? m : 0);
  double* dend = smw_g + (smw ? m : 0);
  // level 0: eight vectors of chunk0 entries, [u | t | xa | xb | y | r | w | 1/diag(L + sigma I)]
  T* base0 = reinterpret_cast<T*>(dend);
  T* u = base0;
  T* t = base0 + chunk0;
  T* xa0 = base0 + 2 * chunk0;
  T* xb0 = base0 + 3 * chunk0;
  T* y = base0 + 4 * chunk0;
  T* r = base0 + 5 * chunk0;
  T* wv = base0 + 6 * chunk0;
  T* di0 = base0 + 7 * chunk0;
  T* lvl = base0 + 8 * chunk0;  // levels >= 1: [xa | xb | rr | tt | dinv] of `chunk` entries each, at G.lev[l].off
  // this CTA's tables: after the vectors in shared memory, or its slice of the global copy
  constexpr bool kF32 = sizeof(T) == sizeof(float);
  char* tbase = G.tab_smem[kF32 ? 0 : 1]
                    ? reinterpret_cast<char*>(((uintptr_t)(lvl + G.lvl_elems) + 15) & ~(uintptr_t)15)
                    : G.tab_glob + (size_t)rank * G.tab_bytes;
  uint32_t* nbA = reinterpret_cast<uint32_t*>(tbase + G.nb_a);
  T* nbC = G.nb_c >= 0 ? reinterpret_cast<T*>(tbase + G.nb_c) : nullptr;
  T* dg0 = reinterpret_cast<T*>(tbase + G.dg);
  T* zw = reinterpret_cast<T*>(scal + 15);  // a zero word: the address of a missing neighbour

  const double lam = A.lam;
  const double c = A.coef[0];
  const double d = A.coef[1];
  const double e = d - c * c;

  for (int a = tid; a < m; a += nth) sS[a] = KIND == 0 ? A.xi[a] * A.xi[a] : A.s[a];
  if (tid == 0) scal[15] = 0.0;
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
  const double sig_now = sqrt(fmax(d + wbar / lam, 1e-12));
  // the v side's correction keeps the shift its cache was formed with while the
  // new one stays within 25 % of it (same inputs in every thread: same decision)
  bool smw_build = false;
  double sigd = sig_now;
  if (smw) {
    const double sref = G.smw_sig[0];
    smw_build = !(G.smw_sig[1] == (double)sizeof(T) && sref > 0.0 && fabs(sig_now / sref - 1.0) <= 0.25);
    if (!smw_build) sigd = sref;
  }
  const T sig = (T)sigd;
  const T om = (T)kOmega;

  // ---- level helpers -------------------------------------------------------------
  auto nown = [&](int l) -> int {
    const DevMgLevel& V = G.lev[l];
    if (!V.dist) return rank == 0 ? V.n : 0;
    return max(0, min(V.n - rank * V.chunk, V.chunk));
  };
  auto gbeg = [&](int l) -> int { return l == 0 ? beg0 : (G.lev[l].dist ? rank * G.lev[l].chunk : 0); };
  auto lbase = [&](int l) -> T* { return l == 0 ? base0 : lvl + G.lev[l].off; };
  // vector k of level l (0 xa, 1 xb, 2 rr, 3 tt, 4 dinv); level 0 keeps its own slots
  auto slot = [&](int l, int k) -> int {
    if (l > 0) return k;
    return k == 0 ? 2 : k == 1 ? 3 : k == 3 ? 1 : 7;
  };
  auto bufs = [&](int l, int k) -> T* {
    const int ch = l == 0 ? chunk0 : G.lev[l].chunk;
    return lbase(l) + slot(l, k) * ch;
  };
  auto boff = [&](int l, int k) -> uint32_t {  // byte offset of vector k from the level's first vector
    const int ch = l == 0 ? chunk0 : G.lev[l].chunk;
    return (uint32_t)(slot(l, k) * ch * (int)sizeof(T));
  };
  // cluster-window address of row `ref` (packed owner/local) of level l's first vector
  auto refaddr = [&](int l, int ref) -> uint32_t {
    return mg_mapa(mg_smem_u32(lbase(l) + (ref & 0xFFFFFF)), (uint32_t)(ref >> 24));
  };
  // lanes per row for a level with `rows` rows in this CTA: rows times lanes fill the CTA
  auto gsize = [&](int rows) -> int {
    int g = 1;
    while (g < 32 && 2 * g * rows <= nth) g *= 2;
    return g;
  };

  // ---- per-launch set-up of the rows this CTA owns --------------------------------
  if (KIND == 0) {
    for (int li = tid; li < n0; li += nth) {
      const int i = beg0 + li;
      double o = 0.0;
      for (int a = 0; a < m; ++a) o += (double)A.Om[i + (int64_t)a * A.ldo] * sS[a];
      A.omt[i] = o;
    }
  }
  const uint32_t zaddr = mg_mapa(mg_smem_u32(zw), (uint32_t)rank);
  for (int li = tid; li < n0; li += nth) {
    const int i = beg0 + li;
    di0[li] = (T)(1.0 / (L.diag[i] + sigd));
    dg0[li] = (T)L.diag[i];
    for (int k = 0; k < L.K; ++k) {
      const int ref = __ldg(L.nbrp + (size_t)k * L.n + i);
      nbA[k * chunk0 + li] = ref >= 0 ? refaddr(0, ref) : zaddr;
      if (nbC) nbC[k * chunk0 + li] = ref >= 0 ? (T)L.offw[(size_t)k * L.n + i] : (T)0;
    }
  }
  // local CSR sections of the rows this CTA owns: row pointer relative to its first row, then entries
  auto fill = [&](int nrows, int gfirst, const int* rp, const int* cp, int lref, int64_t o_rp, int64_t o_a,
                  int64_t o_c, auto&& coef) {
    if (nrows <= 0) return;
    int* lrp = reinterpret_cast<int*>(tbase + o_rp);
    uint32_t* la = reinterpret_cast<uint32_t*>(tbase + o_a);
    T* lc = reinterpret_cast<T*>(tbase + o_c);
    const int q0 = rp[gfirst], q1 = rp[gfirst + nrows];
    for (int li = tid; li <= nrows; li += nth) lrp[li] = rp[gfirst + li] - q0;
    for (int q = q0 + tid; q < q1; q += nth) {  // one thread per entry: coalesced, loads in flight together
      la[q - q0] = refaddr(lref, cp[q]);
      lc[q - q0] = coef(q);
    }
  };
  for (int l = 0; l < G.nlev - 1; ++l) {
    const DevMgLevel& V = G.lev[l];
    const int no = nown(l), gb = gbeg(l);
    if (l >= 1) {
      T* dv = bufs(l, 4);
      for (int li = tid; li < no; li += nth) {
        const double dd = V.dl[gb + li] + sigd * V.dm[gb + li];
        dv[li] = (T)(dd > 0.0 ? 1.0 / dd : 0.0);
      }
      fill(no, gb, V.rp, V.cp, l, V.op_rp, V.op_a, V.op_c, [&](int q) { return (T)(V.lv[q] + sigd * V.mv[q]); });
    }
    fill(no, gb, V.prp, V.pcp, l + 1, V.p_rp, V.p_a, V.p_c, [&](int q) { return (T)V.pv[q]; });
    fill(nown(l + 1), gbeg(l + 1), V.rrp, V.rcp, l, V.r_rp, V.r_a, V.r_c, [&](int q) { return (T)V.rv[q]; });
  }
  __syncthreads();

  // (L + shift I) x on level 0 for row li, x the level-0 vector at byte offset bo from u;
  // up to six neighbours: every address and value load is issued before the first add
  auto lap0 = [&](int li, uint32_t bo, T shift) -> T {
    const T* xv = reinterpret_cast<const T*>(reinterpret_cast<const char*>(base0) + bo);
    T acc = (dg0[li] + shift) * xv[li];
    if (L.K <= 6) {
      uint32_t ad[6];
      T nv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) ad[k] = k < L.K ? nbA[k * chunk0 + li] : zaddr;
#pragma unroll
      for (int k = 0; k < 6; ++k) nv[k] = ad[k] == zaddr ? (T)0 : mg_ld<T>(ad[k] + bo);
      if (nbC) {
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (k < L.K) acc += nbC[k * chunk0 + li] * nv[k];
      } else {
        acc -= ((nv[0] + nv[1]) + (nv[2] + nv[3])) + (nv[4] + nv[5]);
      }
      return acc;
    }
    for (int k = 0; k < L.K; ++k) {
      const uint32_t a = nbA[k * chunk0 + li];
      const T nv = a == zaddr ? (T)0 : mg_ld<T>(a + bo);
      acc += (nbC ? nbC[k * chunk0 + li] : (T)-1) * nv;
    }
    return acc;
  };
  // this lane's share of local table row li: entries lrp[li] + lane, + g, ... < lrp[li + 1]
  auto trow = [&](int64_t o_rp, int64_t o_a, int64_t o_c, int li, int lane, int g, uint32_t bo) -> T {
    const int* lrp = reinterpret_cast<const int*>(tbase + o_rp);
    const uint32_t* la = reinterpret_cast<const uint32_t*>(tbase + o_a);
    const T* lc = reinterpret_cast<const T*>(tbase + o_c);
    T acc = (T)0;
    const int q1 = lrp[li + 1];
    int q = lrp[li] + lane;
    // four entries at a time: addresses, then the four remote values, then the products
    for (; q + 3 * g < q1; q += 4 * g) {
      const uint32_t a0 = la[q], a1 = la[q + g], a2 = la[q + 2 * g], a3 = la[q + 3 * g];
      const T v0 = mg_ld<T>(a0 + bo), v1 = mg_ld<T>(a1 + bo), v2 = mg_ld<T>(a2 + bo), v3 = mg_ld<T>(a3 + bo);
      acc += (lc[q] * v0 + lc[q + g] * v1) + (lc[q + 2 * g] * v2 + lc[q + 3 * g] * v3);
    }
    for (; q < q1; q += g) acc += lc[q] * mg_ld<T>(la[q] + bo);
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
      T sum = li < no ? part(li, lane, g) : (T)0;
      sum = group_sum(sum, g);
      if (li < no && lane == 0) fin(li, sum);
    }
  };
  // (L_l + sigma M_l) x row share on level l, x = vector k of the level
  auto arow = [&](int l, int k) {
    return [&, l, k](int li, int lane, int g) -> T {
      if (l == 0) return lap0(li, boff(0, k), sig);
      const DevMgLevel& V = G.lev[l];
      return trow(V.op_rp, V.op_a, V.op_c, li, lane, g, boff(l, k));
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
    sweep(l, arow(l, 0), [&](int li, T ax) { xb[li] = xa[li] + om * (R[li] - ax) * dv[li]; });
    lsync(l);
    sweep(l, arow(l, 1), [&](int li, T ax) { tt[li] = R[li] - ax; });
    lsync(l);
    // restriction: rows of level l+1 owned here (CTA 0 owns all rows of its levels)
    const DevMgLevel& V = G.lev[l];
    T* rn = bufs(l + 1, 2);
    const uint32_t bo = boff(l, 3);
    sweep(
        l + 1, [&](int lj, int lane, int g) -> T { return trow(V.r_rp, V.r_a, V.r_c, lj, lane, g, bo); },
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
    sweep(
        l,
        [&](int li, int lane, int g) -> T {
          return trow(V.p_rp, V.p_a, V.p_c, li, lane, g, 0u);  // level l+1's xa is its first vector
        },
        [&](int li, T v) { xa[li] = xb[li] + v; });
    lsync(l);
    sweep(l, arow(l, 0), [&](int li, T ax) { xb[li] = xa[li] + om * (R[li] - ax) * dv[li]; });
    lsync(l);
    sweep(l, arow(l, 1), [&](int li, T ax) { OUT[li] = scale * (xb[li] + om * (R[li] - ax) * dv[li]); });
  };
  // exact solve on the coarsest level (CTA 0): x = Q diag(1 / (mu + sigma)) Q^T r, lane groups per entry
  auto coarse = [&]() {
    __syncthreads();  // the restriction into the coarsest level wrote rows of other threads
    T* rc = bufs(G.nlev - 1, 2);
    T* xc = bufs(G.nlev - 1, 0);
    const int g = gsize(nc), rpp = nth / g, lane = tid % g;
    for (int base = 0; base < nc; base += rpp) {
      const int k = base + tid / g;
      double acc = 0.0;
      if (k < nc)
        for (int i = lane; i < nc; i += g) acc += cQ[i + k * nc] * (double)rc[i];
      acc = group_sum(acc, g);
      if (k < nc && lane == 0) ctmp[k] = acc / (fmax(cmu[k], 0.0) + sigd);
    }
    __syncthreads();
    for (int base = 0; base < nc; base += rpp) {
      const int i = base + tid / g;
      double acc = 0.0;
      if (i < nc)
        for (int k = lane; k < nc; k += g) acc += cQ[i + k * nc] * ctmp[k];
      acc = group_sum(acc, g);
      if (i < nc && lane == 0) xc[i] = (T)acc;
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
        double sum = 0.0;
        for (int q = 0; q < C; ++q) sum += cl.map_shared_rank(ypart, (unsigned)q)[a];
        sY[a] = sS[a] * sum;
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
  const uint32_t bo_u = 0u, bo_t = (uint32_t)(chunk0 * (int)sizeof(T));

  // ---- v side: Sherman-Morrison-Woodbury correction for the rank-m data term -----
  // B_hat ~ M0 + X S X^T with M0^-1 = (1 / lam) V(V(.)) and S = D^2 = diag(s):
  //   B^-1 r = y - MX D (I + D X^T MX D)^-1 D X^T y,   y = M0^-1 r,  MX = M0^-1 X.
  T* mx = reinterpret_cast<T*>(G.smw_mx);
  if (smw) {
    if (smw_build) {
      for (int a = 0; a < m; ++a) {
        for (int li = tid; li < n0; li += nth) {  // column a of X on the own rows
          const int i = beg0 + li;
          double xa = 0.0;
          for (int q = A.X.xr_ptr[i]; q < A.X.xr_ptr[i + 1]; ++q)
            if (A.X.xr_col[q] == a) xa += A.X.xr_val[q];
          r[li] = (T)xa;
        }
        vcycle(r, y, (T)1);
        vcycle(y, u, (T)(1.0 / lam));
        for (int li = tid; li < n0; li += nth) mx[(size_t)(beg0 + li) * m + a] = u[li];
      }
      __syncthreads();
      // X^T MX: this CTA's rows, then the cluster's partials in rank order
      for (int idx = tid; idx < m * m; idx += nth) {
        const int a = idx / m, b = idx % m;
        double acc = 0.0;
        for (int q = A.X.lx_ptr[rank * m + a]; q < A.X.lx_ptr[rank * m + a + 1]; ++q)
          acc += A.X.lx_val[q] * (double)mx[(size_t)(beg0 + A.X.lx_row[q]) * m + b];
        smw_part[idx] = acc;
      }
      cl.sync();
      for (int idx = tid; idx < m * m; idx += nth) {
        double acc = 0.0;
        for (int q = 0; q < C; ++q) acc += cl.map_shared_rank(smw_part, (unsigned)q)[idx];
        smw_xx[idx] = acc;
        if (rank == 0) G.smw_xx[idx] = acc;
      }
      if (rank == 0 && tid == 0) {
        G.smw_sig[0] = sigd;
        G.smw_sig[1] = (double)sizeof(T);
      }
    } else {
      for (int idx = tid; idx < m * m; idx += nth) smw_xx[idx] = G.smw_xx[idx];
    }
    __syncthreads();
    // (I + D X^T MX D)^-1 by Gauss-Jordan (symmetric positive definite: no pivoting), in every CTA
    for (int idx = tid; idx < m * m; idx += nth) {
      const int a = idx / m, b = idx % m;
      smw_ci[idx] = (a == b ? 1.0 : 0.0) + sqrt(fmax(sS[a], 0.0)) * smw_xx[idx] * sqrt(fmax(sS[b], 0.0));
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      const double pinv = 1.0 / smw_ci[k * m + k];
      if (tid < m) smw_g[tid] = smw_ci[tid * m + k];  // column k before the step
      __syncthreads();
      if (tid < m) smw_ci[k * m + tid] = (tid == k ? 1.0 : smw_ci[k * m + tid]) * pinv;
      __syncthreads();
      for (int idx = tid; idx < m * m; idx += nth) {
        const int a = idx / m, b = idx % m;
        if (a != k) smw_ci[idx] = (b == k ? 0.0 : smw_ci[idx]) - smw_g[a] * smw_ci[k * m + b];
      }
      __syncthreads();
    }
  }
  // u <- u - MX D C^-1 D X^T u  (u = M0^-1 r on the own rows)
  auto smw_correct = [&]() {
    __syncthreads();  // the V-cycle wrote u one thread per row; X^T u reads rows of other threads
    ypartial(u);
    cl.sync();
    for (int a = tid; a < m; a += nth) {
      double sum = 0.0;
      for (int q = 0; q < C; ++q) sum += cl.map_shared_rank(ypart, (unsigned)q)[a];
      smw_xt[a] = sqrt(fmax(sS[a], 0.0)) * sum;
    }
    __syncthreads();
    for (int a = tid; a < m; a += nth) {
      double acc = 0.0;
      for (int b = 0; b < m; ++b) acc += smw_ci[a * m + b] * smw_xt[b];
      smw_g[a] = sqrt(fmax(sS[a], 0.0)) * acc;
    }
    __syncthreads();
    for (int li = tid; li < n0; li += nth) {
      const T* row = mx + (size_t)(beg0 + li) * m;
      T acc = (T)0;
      for (int b = 0; b < m; ++b) acc += row[b] * (T)smw_g[b];
      u[li] -= acc;
    }
  };

  // r0 = b - A x0
  for (int li = tid; li < n0; li += nth) u[li] = (T)A.x[beg0 + li];
  cl.sync();
  for (int li = tid; li < n0; li += nth) t[li] = lap0(li, bo_u, cT);
  ypartial(u);
  cl.sync();
  gather();
  {
    double v1[1] = {0.0};
    for (int li = tid; li < n0; li += nth) {
      const int i = beg0 + li;
      const T wi = lamT * (lap0(li, bo_t, cT) + eT * u[li]) + data(li, u[li]);
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
      if (smw) smw_correct();
      cl.sync();
      for (int li = tid; li < n0; li += nth) t[li] = lap0(li, bo_u, cT);
      ypartial(u);
      cl.sync();
      gather();
      double v[3] = {0.0, 0.0, 0.0};
      for (int li = tid; li < n0; li += nth) {
        const T ui = u[li];
        const T wi = lamT * (lap0(li, bo_t, cT) + eT * ui) + data(li, ui);
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

size_t mg_smem_bytes(const DevMg& g, int chunk0, int m, bool fp32, bool tables) {
  const size_t tsz = fp32 ? sizeof(float) : sizeof(double);
  const size_t dbl = 8 + 128 + 16 + 3 * (size_t)m + (size_t)g.nc * g.nc + 2 * (size_t)g.nc +
                     (g.smw ? 3 * (size_t)m * m + 2 * (size_t)m : 0);
  const size_t base = sizeof(double) * dbl + tsz * (8 * (size_t)chunk0 + (size_t)g.lvl_elems) + 16;
  return tables ? base + 16 + (size_t)g.tab_bytes : base;
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
