// Learned preconditioner network: 4 layers of 3x3x3 convolutions on the voxel
// box (channels 2 -> 16 -> 16 -> 16 -> 1, zero padding, ReLU between layers),
// BF16 weights and activations, float32 accumulation, float32 gradients and
// Adam state.  Forward, backward (data and weight) and the optimiser step are
// hand-written kernels; reductions are fixed-order (one block per weight
// group, then a fixed tree), so training is reproducible.
//
// Input channels: 0 = Jacobi-scaled residual D^-1 r / s on the mask voxels,
// 1 = the mask.  The solver uses z = D^-1 r + s * net(input) (cr_api.cu).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "conreg.h"
#include "cr_common.cuh"

namespace cr {
void set_global_error(const std::string& msg);  // cr_api.cu
}

namespace {

using bf16 = __nv_bfloat16;
constexpr int kL = 4;
constexpr int kCh[kL + 1] = {2, 16, 16, 16, 1};
constexpr int kThreads = 256;

struct Dims {
  int D, H, W;
  int64_t V;
};

__device__ __forceinline__ bool nb(const Dims& g, int z, int y, int x, int t, int64_t& off) {
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int zz = z + dz, yy = y + dy, xx = x + dx;
  if (zz < 0 || zz >= g.D || yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return false;
  off = ((int64_t)zz * g.H + yy) * g.W + xx;
  return true;
}

// Storage type S (bf16 on the solver path, double in the float64 check) and
// accumulation type A (float, double).
__device__ __forceinline__ float to_acc(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_acc(double v) { return v; }
template <class S>
__device__ __forceinline__ S from_acc(float v);
template <>
__device__ __forceinline__ bf16 from_acc<bf16>(float v) {
  return __float2bfloat16_rn(v);
}
template <class S>
__device__ __forceinline__ S from_acc(double v) {
  return v;
}
__device__ __forceinline__ float fmax0(float v) { return fmaxf(v, 0.f); }
__device__ __forceinline__ double fmax0(double v) { return fmax(v, 0.0); }

// Weights as A: staged in shared memory for float accumulation, read from
// global memory in the float64 check (a 16 x 16 x 27 double block exceeds the
// static shared-memory limit).
// out[b, co, v] = act(bias[co] + sum_ci sum_t W[co, ci, t] in[b, ci, v + t])
template <int CI, int CO, bool RELU, bool OUTA, class S, class A>
__global__ void __launch_bounds__(kThreads) conv_fwd(Dims g, int B, const S* __restrict__ in,
                                                     const S* __restrict__ Wb, const A* __restrict__ bias,
                                                     void* out) {
  __shared__ float Wsf[sizeof(A) == 4 ? CO * CI * 27 : 1];
  const A* Ws;
  if constexpr (sizeof(A) == 4) {
    for (int i = threadIdx.x; i < CO * CI * 27; i += blockDim.x) Wsf[i] = to_acc(Wb[i]);
    __syncthreads();
    Ws = reinterpret_cast<const A*>(Wsf);
  } else {
    Ws = reinterpret_cast<const A*>(Wb);
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * g.V) return;
  const int b = (int)(t / g.V);
  const int64_t v = t % g.V;
  const int x = (int)(v % g.W), y = (int)((v / g.W) % g.H), z = (int)(v / ((int64_t)g.W * g.H));
  A acc[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = bias[co];
  const S* ib = in + (int64_t)b * CI * g.V;
  for (int tap = 0; tap < 27; ++tap) {
    int64_t off;
    if (!nb(g, z, y, x, tap, off)) continue;
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) {
      const A a = to_acc(ib[(int64_t)ci * g.V + off]);
#pragma unroll
      for (int co = 0; co < CO; ++co) acc[co] = fma(Ws[(co * CI + ci) * 27 + tap], a, acc[co]);
    }
  }
#pragma unroll
  for (int co = 0; co < CO; ++co) {
    const A r = RELU ? fmax0(acc[co]) : acc[co];
    if (OUTA)
      ((A*)out)[((int64_t)b * CO + co) * g.V + v] = r;
    else
      ((S*)out)[((int64_t)b * CO + co) * g.V + v] = from_acc<S>(r);
  }
}

// gin[b, ci, u] = relu'(a_in[b, ci, u]) * sum_co sum_t W[co, ci, t] gout[b, co, u - t]
template <int CI, int CO, class S, class A>
__global__ void __launch_bounds__(kThreads) conv_bwd_data(Dims g, int B, const A* __restrict__ gout,
                                                          const S* __restrict__ Wb, const S* __restrict__ ain,
                                                          A* __restrict__ gin) {
  __shared__ float Wsf[sizeof(A) == 4 ? CO * CI * 27 : 1];
  const A* Ws;
  if constexpr (sizeof(A) == 4) {
    for (int i = threadIdx.x; i < CO * CI * 27; i += blockDim.x) Wsf[i] = to_acc(Wb[i]);
    __syncthreads();
    Ws = reinterpret_cast<const A*>(Wsf);
  } else {
    Ws = reinterpret_cast<const A*>(Wb);
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * g.V) return;
  const int b = (int)(t / g.V);
  const int64_t u = t % g.V;
  const int x = (int)(u % g.W), y = (int)((u / g.W) % g.H), z = (int)(u / ((int64_t)g.W * g.H));
  A acc[CI];
#pragma unroll
  for (int ci = 0; ci < CI; ++ci) acc[ci] = (A)0;
  const A* gb = gout + (int64_t)b * CO * g.V;
  for (int tap = 0; tap < 27; ++tap) {
    int64_t off;
    if (!nb(g, z, y, x, 26 - tap, off)) continue;  // v = u - t  <=>  tap mirrored
#pragma unroll
    for (int co = 0; co < CO; ++co) {
      const A gv = gb[(int64_t)co * g.V + off];
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) acc[ci] = fma(Ws[(co * CI + ci) * 27 + tap], gv, acc[ci]);
    }
  }
#pragma unroll
  for (int ci = 0; ci < CI; ++ci) {
    const int64_t o = ((int64_t)b * CI + ci) * g.V + u;
    gin[o] = to_acc(ain[o]) > (A)0 ? acc[ci] : (A)0;
  }
}

// dW[co, ci, t] = sum_b sum_v gout[b, co, v] a_in[b, ci, v + t]; db[co] = sum_b sum_v gout[b, co, v]
// one block per (co, ci); fixed-order block reduction
template <int CI, int CO, class S, class A>
__global__ void __launch_bounds__(kThreads) conv_bwd_weight(Dims g, int B, const A* __restrict__ gout,
                                                            const S* __restrict__ ain, A* __restrict__ dW,
                                                            A* __restrict__ db) {
  const int co = blockIdx.x / CI, ci = blockIdx.x % CI;
  A acc[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) acc[k] = (A)0;
  const int64_t tot = (int64_t)B * g.V;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    const int b = (int)(t / g.V);
    const int64_t v = t % g.V;
    const A gv = gout[((int64_t)b * CO + co) * g.V + v];
    if (gv == (A)0) continue;
    const int x = (int)(v % g.W), y = (int)((v / g.W) % g.H), z = (int)(v / ((int64_t)g.W * g.H));
    const S* ab = ain + ((int64_t)b * CI + ci) * g.V;
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) {
      int64_t off;
      if (nb(g, z, y, x, tap, off)) acc[tap] = fma(gv, to_acc(ab[off]), acc[tap]);
    }
    acc[27] += gv;
  }
  __shared__ A red[kThreads / 32][28];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 28; ++k) {
    A s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < 28) {
    A s = (A)0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    if (threadIdx.x < 27)
      dW[(co * CI + ci) * 27 + threadIdx.x] = s;
    else if (ci == 0)
      db[co] = s;
  }
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ x, bf16* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// partial sums of num = sum m (o - t)^2, den = sum m t^2 over blocks (fixed order)
template <class A>
__global__ void loss_partial_kernel(int64_t V, int B, const A* __restrict__ out, const A* __restrict__ tgt,
                                    const uint8_t* __restrict__ mask, A* __restrict__ part) {
  A a = (A)0, c = (A)0;
  const int64_t tot = (int64_t)B * V;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[t % V]) continue;
    const A d = out[t] - tgt[t];
    a = fma(d, d, a);
    c = fma(tgt[t], tgt[t], c);
  }
  __shared__ A red[2][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    A s0 = (A)0, s1 = (A)0;
    for (int w = 0; w < kThreads / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

template <class A>
__global__ void loss_final_kernel(int nb, const A* __restrict__ part, A* __restrict__ res) {
  if (threadIdx.x == 0) {
    A a = (A)0, c = (A)0;
    for (int b = 0; b < nb; ++b) {
      a += part[2 * b];
      c += part[2 * b + 1];
    }
    res[0] = a;
    res[1] = c;
    res[2] = c > (A)0 ? a / c : (A)0;
  }
}

// g = 2 m (o - t) / den
template <class A>
__global__ void loss_grad_kernel(int64_t V, int B, const A* __restrict__ out, const A* __restrict__ tgt,
                                 const uint8_t* __restrict__ mask, const A* __restrict__ res, A* __restrict__ g) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * V) return;
  const A den = res[1];
  g[t] = (mask[t % V] && den > (A)0) ? (A)2 * (out[t] - tgt[t]) / den : (A)0;
}

__global__ void adam_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

struct cr_net {
  Dims g{};
  int Bcap = 0;
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;
  float *W[kL] = {}, *b[kL] = {}, *gW[kL] = {}, *gb[kL] = {}, *mW[kL] = {}, *vW[kL] = {}, *mb[kL] = {},
        *vb[kL] = {};
  bf16* Wb[kL] = {};
  bf16* act[kL] = {};   // act[0] = input (B x 2 x V), act[l] = output of layer l (l = 1..3)
  float* out = nullptr; // B x V
  float *g0 = nullptr, *g1 = nullptr;  // gradient ping-pong (B x 16 x V)
  float* part = nullptr;
  float* res = nullptr;
  int step = 0;
};

namespace {

int64_t wcount(int l) { return (int64_t)kCh[l + 1] * kCh[l] * 27; }

template <class T>
bool net_alloc(cr_net* n, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), n->st);
  n->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

// The network's device buffers for one instantiation (S storage, A accumulation).
template <class S, class A>
struct NetBufs {
  const S* Wb[kL];
  const A* b[kL];
  S* act[kL];    // act[0] = input (B x 2 x V), act[l] = output of layer l (l = 1..3)
  A* out;        // B x V
  A *g0, *g1;    // gradient ping-pong (B x 16 x V)
  A *part, *res;
  A *gW[kL], *gb[kL];
};

template <class S, class A>
void launch_fwd(const NetBufs<S, A>& n, const Dims& g, int B, cudaStream_t st) {
  const unsigned grid = nblk((int64_t)B * g.V);
  cr::count_launch();
  conv_fwd<2, 16, true, false, S, A><<<grid, kThreads, 0, st>>>(g, B, n.act[0], n.Wb[0], n.b[0], n.act[1]);
  cr::count_launch();
  conv_fwd<16, 16, true, false, S, A><<<grid, kThreads, 0, st>>>(g, B, n.act[1], n.Wb[1], n.b[1], n.act[2]);
  cr::count_launch();
  conv_fwd<16, 16, true, false, S, A><<<grid, kThreads, 0, st>>>(g, B, n.act[2], n.Wb[2], n.b[2], n.act[3]);
  cr::count_launch();
  conv_fwd<16, 1, false, true, S, A><<<grid, kThreads, 0, st>>>(g, B, n.act[3], n.Wb[3], n.b[3], n.out);
}

// loss + gradients of all parameters into gW/gb for the batch in act[0]/out
template <class S, class A>
void launch_bwd(const NetBufs<S, A>& n, const Dims& g, int B, const A* tgt, const uint8_t* mask, cudaStream_t st) {
  const unsigned grid = nblk((int64_t)B * g.V);
  const int nbp = 128;
  cr::count_launch();
  loss_partial_kernel<A><<<nbp, kThreads, 0, st>>>(g.V, B, n.out, tgt, mask, n.part);
  cr::count_launch();
  loss_final_kernel<A><<<1, 32, 0, st>>>(nbp, n.part, n.res);
  cr::count_launch();
  loss_grad_kernel<A><<<grid, kThreads, 0, st>>>(g.V, B, n.out, tgt, mask, n.res, n.g0);
  // layer 3 (16 -> 1, linear): g0 = dloss/dz_3
  cr::count_launch();
  conv_bwd_weight<16, 1, S, A><<<16, kThreads, 0, st>>>(g, B, n.g0, n.act[3], n.gW[3], n.gb[3]);
  cr::count_launch();
  conv_bwd_data<16, 1, S, A><<<grid, kThreads, 0, st>>>(g, B, n.g0, n.Wb[3], n.act[3], n.g1);
  cr::count_launch();
  conv_bwd_weight<16, 16, S, A><<<256, kThreads, 0, st>>>(g, B, n.g1, n.act[2], n.gW[2], n.gb[2]);
  cr::count_launch();
  conv_bwd_data<16, 16, S, A><<<grid, kThreads, 0, st>>>(g, B, n.g1, n.Wb[2], n.act[2], n.g0);
  cr::count_launch();
  conv_bwd_weight<16, 16, S, A><<<256, kThreads, 0, st>>>(g, B, n.g0, n.act[1], n.gW[1], n.gb[1]);
  cr::count_launch();
  conv_bwd_data<16, 16, S, A><<<grid, kThreads, 0, st>>>(g, B, n.g0, n.Wb[1], n.act[1], n.g1);
  cr::count_launch();
  conv_bwd_weight<2, 16, S, A><<<32, kThreads, 0, st>>>(g, B, n.g1, n.act[0], n.gW[0], n.gb[0]);
}

NetBufs<bf16, float> bufs(const cr_net* n) {
  NetBufs<bf16, float> b{};
  for (int l = 0; l < kL; ++l) {
    b.Wb[l] = n->Wb[l];
    b.b[l] = n->b[l];
    b.act[l] = n->act[l];
    b.gW[l] = n->gW[l];
    b.gb[l] = n->gb[l];
  }
  b.out = n->out;
  b.g0 = n->g0;
  b.g1 = n->g1;
  b.part = n->part;
  b.res = n->res;
  return b;
}

void launch_fwd(cr_net* n, int B) { launch_fwd(bufs(n), n->g, B, n->st); }
void launch_bwd(cr_net* n, int B, const float* tgt, const uint8_t* mask) {
  launch_bwd(bufs(n), n->g, B, tgt, mask, n->st);
}

void refresh_bf16(cr_net* n) {
  for (int l = 0; l < kL; ++l) {
    cr::count_launch();
    to_bf16_kernel<<<nblk(wcount(l)), kThreads, 0, n->st>>>(wcount(l), n->W[l], n->Wb[l]);
  }
}

void load_input(cr_net* n, int B, const float* in) {
  cr::count_launch();
  to_bf16_kernel<<<nblk((int64_t)B * 2 * n->g.V), kThreads, 0, n->st>>>((int64_t)B * 2 * n->g.V, in, n->act[0]);
}

}  // namespace

extern "C" {

int64_t cr_net_param_count(void) {
  int64_t c = 0;
  for (int l = 0; l < kL; ++l) c += wcount(l) + kCh[l + 1];
  return c;
}

cr_status cr_net_create(int32_t D, int32_t H, int32_t W, int32_t batch_cap, uint64_t seed, void* stream,
                        cr_net** out) {
  if (out) *out = nullptr;
  if (!out || D < 1 || H < 1 || W < 1 || batch_cap < 1 || (int64_t)D * H * W > (1ll << 26)) {
    cr::set_global_error("cr_net_create: bad dimensions or batch capacity");
    return CR_EINVAL;
  }
  cr_net* n = new cr_net();
  n->g = Dims{D, H, W, (int64_t)D * H * W};
  n->Bcap = batch_cap;
  n->st = (cudaStream_t)stream;
  bool ok = true;
  const int64_t V = n->g.V;
  for (int l = 0; l < kL && ok; ++l) {
    ok = ok && net_alloc(n, &n->W[l], wcount(l)) && net_alloc(n, &n->b[l], kCh[l + 1]) &&
         net_alloc(n, &n->gW[l], wcount(l)) && net_alloc(n, &n->gb[l], kCh[l + 1]) &&
         net_alloc(n, &n->mW[l], wcount(l)) && net_alloc(n, &n->vW[l], wcount(l)) &&
         net_alloc(n, &n->mb[l], kCh[l + 1]) && net_alloc(n, &n->vb[l], kCh[l + 1]) &&
         net_alloc(n, &n->Wb[l], wcount(l)) && net_alloc(n, &n->act[l], (size_t)batch_cap * kCh[l] * V);
  }
  ok = ok && net_alloc(n, &n->out, (size_t)batch_cap * V) && net_alloc(n, &n->g0, (size_t)batch_cap * 16 * V) &&
       net_alloc(n, &n->g1, (size_t)batch_cap * 16 * V) && net_alloc(n, &n->part, 256) && net_alloc(n, &n->res, 4);
  if (!ok) {
    cr::set_global_error("cr_net_create: device allocation failed");
    cr_net_destroy(n);
    return CR_ENOMEM;
  }
  // He-style initialisation (seeded); the last layer starts at zero so the
  // untrained preconditioner is exactly Jacobi
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (int l = 0; l < kL; ++l) {
    std::vector<float> w(wcount(l));
    const float sc = l == kL - 1 ? 0.f : std::sqrt(2.f / (27.f * kCh[l]));
    for (auto& x : w) x = sc * nd(rng);
    cudaMemcpyAsync(n->W[l], w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, n->st);
  }
  refresh_bf16(n);
  if (cudaStreamSynchronize(n->st) != cudaSuccess) {
    cudaGetLastError();
    cr::set_global_error("cr_net_create: CUDA error");
    cr_net_destroy(n);
    return CR_ECUDA;
  }
  *out = n;
  return CR_OK;
}

void cr_net_destroy(cr_net* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st);
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

cr_status cr_net_get_params(cr_net* n, float* host, int64_t count) {
  if (!n || !host || count != cr_net_param_count()) return CR_EINVAL;
  float* h = host;
  for (int l = 0; l < kL; ++l) {
    cudaMemcpyAsync(h, n->W[l], wcount(l) * sizeof(float), cudaMemcpyDeviceToHost, n->st);
    h += wcount(l);
    cudaMemcpyAsync(h, n->b[l], kCh[l + 1] * sizeof(float), cudaMemcpyDeviceToHost, n->st);
    h += kCh[l + 1];
  }
  return cudaStreamSynchronize(n->st) == cudaSuccess ? CR_OK : CR_ECUDA;
}

cr_status cr_net_set_params(cr_net* n, const float* host, int64_t count) {
  if (!n || !host || count != cr_net_param_count()) return CR_EINVAL;
  for (int64_t i = 0; i < count; ++i)
    if (!std::isfinite(host[i])) {
      cr::set_global_error("cr_net_set_params: non-finite parameter");
      return CR_EINVAL;
    }
  const float* h = host;
  for (int l = 0; l < kL; ++l) {
    cudaMemcpyAsync(n->W[l], h, wcount(l) * sizeof(float), cudaMemcpyHostToDevice, n->st);
    h += wcount(l);
    cudaMemcpyAsync(n->b[l], h, kCh[l + 1] * sizeof(float), cudaMemcpyHostToDevice, n->st);
    h += kCh[l + 1];
  }
  refresh_bf16(n);
  return cudaStreamSynchronize(n->st) == cudaSuccess ? CR_OK : CR_ECUDA;
}

cr_status cr_net_forward(cr_net* n, int32_t B, const float* in_dev, float* out_dev) {
  if (!n || !in_dev || !out_dev || B < 1 || B > n->Bcap) return CR_EINVAL;
  load_input(n, B, in_dev);
  launch_fwd(n, B);
  if (cudaMemcpyAsync(out_dev, n->out, (size_t)B * n->g.V * sizeof(float), cudaMemcpyDeviceToDevice, n->st) !=
      cudaSuccess)
    return CR_ECUDA;
  return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ECUDA;
}

cr_status cr_net_gradients(cr_net* n, int32_t B, const float* in_dev, const float* target_dev,
                           const uint8_t* mask_dev, float* loss_host, float* grad_host) {
  if (!n || !in_dev || !target_dev || !mask_dev || B < 1 || B > n->Bcap) return CR_EINVAL;
  load_input(n, B, in_dev);
  launch_fwd(n, B);
  launch_bwd(n, B, target_dev, mask_dev);
  float res[3] = {0, 0, 0};
  cudaMemcpyAsync(res, n->res, sizeof(res), cudaMemcpyDeviceToHost, n->st);
  if (grad_host) {
    float* h = grad_host;
    for (int l = 0; l < kL; ++l) {
      cudaMemcpyAsync(h, n->gW[l], wcount(l) * sizeof(float), cudaMemcpyDeviceToHost, n->st);
      h += wcount(l);
      cudaMemcpyAsync(h, n->gb[l], kCh[l + 1] * sizeof(float), cudaMemcpyDeviceToHost, n->st);
      h += kCh[l + 1];
    }
  }
  if (cudaStreamSynchronize(n->st) != cudaSuccess) return CR_ECUDA;
  if (loss_host) *loss_host = res[2];
  return CR_OK;
}

cr_status cr_net_train_step(cr_net* n, int32_t B, const float* in_dev, const float* target_dev,
                            const uint8_t* mask_dev, float lr, float* loss_host) {
  if (!n || !in_dev || !target_dev || !mask_dev || B < 1 || B > n->Bcap || !(lr > 0.f)) return CR_EINVAL;
  load_input(n, B, in_dev);
  launch_fwd(n, B);
  launch_bwd(n, B, target_dev, mask_dev);
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  for (int l = 0; l < kL; ++l) {
    cr::count_launch();
    adam_kernel<<<nblk(wcount(l)), kThreads, 0, n->st>>>(wcount(l), n->W[l], n->gW[l], n->mW[l], n->vW[l], lr, b1, b2,
                                                        c1, c2, 1e-8f);
    cr::count_launch();
    adam_kernel<<<1, kThreads, 0, n->st>>>(kCh[l + 1], n->b[l], n->gb[l], n->mb[l], n->vb[l], lr, b1, b2, c1, c2,
                                           1e-8f);
  }
  refresh_bf16(n);
  if (loss_host) {
    float res[3];
    cudaMemcpyAsync(res, n->res, sizeof(res), cudaMemcpyDeviceToHost, n->st);
    if (cudaStreamSynchronize(n->st) != cudaSuccess) return CR_ECUDA;
    *loss_host = res[2];
  }
  return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ECUDA;
}

cr_status cr_net_check_f64(int32_t D, int32_t H, int32_t W, int32_t B, const double* params, const double* in,
                           const double* target, const uint8_t* mask, double* out, double* loss, double* grads) {
  if (D < 1 || H < 1 || W < 1 || B < 1 || (int64_t)D * H * W * B > (1ll << 22) || !params || !in || !target ||
      !mask || !out || !loss || !grads) {
    cr::set_global_error("cr_net_check_f64: bad arguments");
    return CR_EINVAL;
  }
  const Dims g{D, H, W, (int64_t)D * H * W};
  const int64_t V = g.V;
  // one device block: parameters and gradients, activations, output, work
  const int64_t np = cr_net_param_count();
  int64_t nact = 0;
  for (int l = 0; l < kL; ++l) nact += (int64_t)B * kCh[l] * V;
  const int64_t total = 2 * np + nact + (int64_t)B * V * 2 + 2 * (int64_t)B * 16 * V + 256 + 4;
  double* blk = nullptr;
  uint8_t* dmask = nullptr;
  cudaStream_t st = nullptr;
  cr_status rc = CR_OK;
  if (cudaMalloc(&blk, sizeof(double) * total) != cudaSuccess || cudaMalloc(&dmask, V) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cr::set_global_error("cr_net_check_f64: device allocation failed");
    rc = CR_ENOMEM;
  } else {
    NetBufs<double, double> b{};
    double* q = blk;
    double* P = q;  // parameters, packed as in cr_net_get_params
    q += np;
    double* Gp = q;  // gradients, same packing
    q += np;
    {
      double *p = P, *gp = Gp;
      for (int l = 0; l < kL; ++l) {
        b.Wb[l] = p;
        b.gW[l] = gp;
        p += wcount(l);
        gp += wcount(l);
        b.b[l] = p;
        b.gb[l] = gp;
        p += kCh[l + 1];
        gp += kCh[l + 1];
      }
    }
    for (int l = 0; l < kL; ++l) {
      b.act[l] = q;
      q += (int64_t)B * kCh[l] * V;
    }
    b.out = q;
    q += (int64_t)B * V;
    double* tg = q;
    q += (int64_t)B * V;
    b.g0 = q;
    q += (int64_t)B * 16 * V;
    b.g1 = q;
    q += (int64_t)B * 16 * V;
    b.part = q;
    q += 256;
    b.res = q;
    cudaMemsetAsync(blk, 0, sizeof(double) * total, st);
    cudaMemcpyAsync(P, params, sizeof(double) * np, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(b.act[0], in, sizeof(double) * B * 2 * V, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(tg, target, sizeof(double) * B * V, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dmask, mask, V, cudaMemcpyHostToDevice, st);
    launch_fwd(b, g, B, st);
    launch_bwd(b, g, B, tg, dmask, st);
    double res[3] = {0, 0, 0};
    cudaMemcpyAsync(out, b.out, sizeof(double) * B * V, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(grads, Gp, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(res, b.res, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      cr::set_global_error("cr_net_check_f64: CUDA error");
      rc = CR_ECUDA;
    } else {
      *loss = res[2];
    }
  }
  if (st) cudaStreamDestroy(st);
  if (blk) cudaFree(blk);
  if (dmask) cudaFree(dmask);
  return rc;
}

}  // extern "C"

namespace cr {
// forward pass on an input already in the network's input buffer layout (B = 1),
// used by the solver's flexible CG: in (2 x V float32) -> out (V float32, device)
cudaError_t net_apply(cr_net* n, const float* in, float* out, cudaStream_t st) {
  cudaStream_t keep = n->st;
  n->st = st;
  load_input(n, 1, in);
  launch_fwd(n, 1);
  n->st = keep;
  return cudaMemcpyAsync(out, n->out, n->g.V * sizeof(float), cudaMemcpyDeviceToDevice, st);
}
int64_t net_voxels(const cr_net* n) { return n->g.V; }
}  // namespace cr
