// Post-processing of a greedy solution W = U Z V^T: one tiled float64 pass
// that forms W on chip (64 x 64 tiles, never the whole ny x nx matrix),
// optionally projects it onto the nonnegative orthant (Sec. 4, dropping the
// nonnegativity constraint), compares it with a reference W* = U* Z* V*^T
// (the error measures of Sec. 3) and keeps eight statistics per CTA.  A
// persistent grid walks the tiles in a fixed order and a single block adds
// the CTAs' statistics in a fixed order, so the results are reproducible bit
// for bit.  The pass is bound by float64 FMA throughput: 2 (j + j*) flops per
// entry of W against 8 bytes per entry when W is written out.
#include <algorithm>

#include "cr_common.cuh"

namespace cr {

namespace {

constexpr int PT = 64;   // output tile edge
constexpr int PK = 16;   // reduction step staged in shared memory
constexpr int PTHREADS = 256;

__device__ __forceinline__ double stat_op(int q, double a, double b) {
  if (q == PS_MIN) return fmin(a, b);
  if (q == PS_MAX || q == PS_MAXABS) return fmax(a, b);
  return a + b;
}

__device__ __forceinline__ double stat_identity(int q) {
  if (q == PS_MIN) return INFINITY;
  if (q == PS_MAX) return -INFINITY;
  return 0.0;
}

// fixed-order block combination of per-thread statistics; thread 0 writes out[0..PS_N)
__device__ void block_stats(double (&v)[PS_N], double* out) {
  __shared__ double scr[PTHREADS / 32][PS_N];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < PS_N; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = stat_op(q, v[q], __shfl_down_sync(0xffffffffu, v[q], o));
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < PS_N; ++q) scr[wid][q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < PS_N; ++q) {
      double a = scr[0][q];
      for (int w = 1; w < nw; ++w) a = stat_op(q, a, scr[w][q]);
      out[q] = a;
    }
}

// acc[a][b] += sum_k P(i0 + tx + 16a, k) V(c0 + ty + 16b, k), k < K; P col-major (ld ldp),
// V(c, k) at V[c + k * ldv].  Rows or columns past the matrix read as zero.
__device__ __forceinline__ void tile_product(int nrow, int ncol, int K, const double* __restrict__ P, int64_t ldp,
                                             const double* __restrict__ V, int64_t ldv, int i0, int c0,
                                             double (*Ps)[PT], double (*Vs)[PT], double (&acc)[4][4]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += PK) {
    // 64 x 16 panels of P and V: 1,024 entries each, four per thread, along the
    // matrices' contiguous (row) index
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int f = tid + e * PTHREADS, r = f & (PT - 1), kq = f >> 6;
      const int k = k0 + kq;
      Ps[kq][r] = (i0 + r < nrow && k < K) ? P[(int64_t)(i0 + r) + (int64_t)k * ldp] : 0.0;
      Vs[kq][r] = (c0 + r < ncol && k < K) ? V[(int64_t)(c0 + r) + (int64_t)k * ldv] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PK; ++q) {
      double pv[4], vv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) pv[a] = Ps[q][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) vv[b] = Vs[q][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(pv[a], vv[b], acc[a][b]);
    }
    __syncthreads();
  }
}

// Columns [col0, col0 + ncols) of W = P V^T (P = U Z, ny x j) against W* = Pr Vr^T.
// Tile t (row-tile fastest) belongs to CTA t mod gridDim.x.  out (may be null)
// receives P(W) for the columns of this launch, column c at out + (c - col0) * ldo.
// part[blockIdx.x * PS_N + q] receives the CTA's statistics.
__global__ void __launch_bounds__(PTHREADS) post_tile_kernel(int ny, int j, const double* __restrict__ P,
                                                             int64_t ldp, const double* __restrict__ V, int64_t ldv,
                                                             int jr, const double* __restrict__ Pr, int64_t ldpr,
                                                             const double* __restrict__ Vr, int64_t ldvr, int nonneg,
                                                             int col0, int ncols, double* __restrict__ out,
                                                             int64_t ldo, double* __restrict__ part) {
  __shared__ double Ps[PK][PT];
  __shared__ double Vs[PK][PT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int rt = (ny + PT - 1) / PT, ct = (ncols + PT - 1) / PT;
  const int64_t ntiles = (int64_t)rt * ct;
  const int cend = col0 + ncols;
  double s[PS_N];
#pragma unroll
  for (int q = 0; q < PS_N; ++q) s[q] = stat_identity(q);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (int)(t % rt) * PT, c0 = col0 + (int)(t / rt) * PT;
    double acc[4][4], accr[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = accr[a][b] = 0.0;
    tile_product(ny, cend, j, P, ldp, V, ldv, i0, c0, Ps, Vs, acc);
    if (jr > 0) tile_product(ny, cend, jr, Pr, ldpr, Vr, ldvr, i0, c0, Ps, Vs, accr);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + ty + 16 * b;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = i0 + tx + 16 * a;
        if (i >= ny || c >= cend) continue;
        const double w = acc[a][b], wr = accr[a][b];
        if (w < 0.0) {
          s[PS_NNEG] += 1.0;
          s[PS_NEG2] = fma(w, w, s[PS_NEG2]);
        }
        s[PS_MIN] = fmin(s[PS_MIN], w);
        s[PS_MAX] = fmax(s[PS_MAX], w);
        s[PS_W2] = fma(w, w, s[PS_W2]);
        const double pw = (nonneg && w < 0.0) ? 0.0 : w;
        const double d = pw - wr;
        s[PS_REF2] = fma(wr, wr, s[PS_REF2]);
        s[PS_DIFF2] = fma(d, d, s[PS_DIFF2]);
        s[PS_MAXABS] = fmax(s[PS_MAXABS], fabs(d));
        if (out) out[(int64_t)i + (int64_t)(c - col0) * ldo] = pw;
      }
    }
  }
  block_stats(s, part + (int64_t)blockIdx.x * PS_N);
}

// out[q] = the combination of part[p * PS_N + q] over p < nparts, in a fixed order
__global__ void post_reduce_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  double s[PS_N];
#pragma unroll
  for (int q = 0; q < PS_N; ++q) s[q] = stat_identity(q);
  for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
    for (int q = 0; q < PS_N; ++q) s[q] = stat_op(q, s[q], part[(int64_t)p * PS_N + q]);
  block_stats(s, out);
}

}  // namespace

int post_blocks() {
  // resident CTAs on the whole GPU (one device per process); initialised once, thread-safe
  static const int nb = [] {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, post_tile_kernel, PTHREADS, 0);
    return std::max(1, sms) * std::max(1, per_sm);
  }();
  return nb;
}

int post_tiles_parts(int ny, int ncols) {
  const int64_t ntiles = (int64_t)((ny + PT - 1) / PT) * ((ncols + PT - 1) / PT);
  return (int)std::min<int64_t>(post_blocks(), std::max<int64_t>(ntiles, 1));
}

void post_tiles(int ny, int j, const double* P, int64_t ldp, const double* V, int64_t ldv, int jr,
                const double* Pr, int64_t ldpr, const double* Vr, int64_t ldvr, int nonneg, int col0, int ncols,
                double* out, int64_t ldo, double* part, cudaStream_t st) {
  const int nb = post_tiles_parts(ny, ncols);
  count_launch();
  post_tile_kernel<<<nb, PTHREADS, 0, st>>>(ny, j, P, ldp, V, ldv, jr, Pr, ldpr, Vr, ldvr, nonneg, col0, ncols,
                                            out, ldo, part);
}

void post_reduce(int nparts, const double* part, double* out, cudaStream_t st) {
  count_launch();
  post_reduce_kernel<<<1, PTHREADS, 0, st>>>(nparts, part, out);
}

}  // namespace cr
