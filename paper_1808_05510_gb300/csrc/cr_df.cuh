// Double-float arithmetic shared by the float32 kernels (see cr_pcg.cu).
#pragma once

#include <cuda_runtime.h>

namespace cr {

// Double-float ("DF") arithmetic: a value is hi + lo with two float32 words,
// about 48 significant bits.  GB300 executes float64 at a small fraction of
// its float32 rate (a dependent float64 add costs ~67 cycles, a divide ~600,
// measured), so the float32 kernel keeps its inner products and CG scalars in
// DF: exact products via FMA (two-product), error-free sums (two-sum), and a
// Newton-corrected quotient.  The sum order is fixed, as in the float64 path.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_prod(float a, float b) {
  const float p = a * b;
  return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;
  return DF{h, e - (h - s)};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float h = p + e;
  return DF{h, e - (h - p)};
}

__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = a.hi / b.hi;
  const DF r = df_sub(a, df_mul(b, DF{q1, 0.f}));
  const float q2 = r.hi / b.hi;
  const float h = q1 + q2;
  return DF{h, q2 - (h - q1)};
}

__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF t;
    t.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    t.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    v = df_add(v, t);
  }
  return v;
}

// Sum NV per-thread DF values over the CTA; thread 0 stores them in out[].
template <int NV>
__device__ __forceinline__ void block_sum_df(DF (&v)[NV], DF* scr, DF* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum_df(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) scr[wid * NV + q] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      DF t = lane < nw ? scr[lane * NV + q] : DF{0.f, 0.f};
      t = warp_sum_df(t);
      if (lane == 0) out[q] = t;
    }
  }
}


}  // namespace cr
