// sd_predictor.cu -- retention-count predictor for batch planning.
//
// A 1-D convolutional network over codon positions predicts, for every codon
// position k and span band s, log1p of the number of retained multiloop
// candidates (Eq. candidates) whose right endpoint lies in codon k and whose
// span falls in band s (spans 5-7, 8-15, ..., 256-511, >= 512).  The plan uses
// the prediction to reserve room for the candidate lists; it never decides
// which candidate is kept (the exact test B < P_S does that), and a list that
// outgrows its room makes the plan repeat the run with worst-case room.
//
// Network: 4 convolutions of width 5 ("same" padding, zero beyond the protein),
// 32 -> 128 -> 128 -> 128 -> 8 channels, ReLU after the first three.  Weights
// and activations are BF16, every contraction accumulates in FP32 on the
// tensor cores (mma.sync m16n8k16 BF16), gradients and the Adam master
// weights are FP32.  Each convolution is an implicit GEMM whose operand
// tiles are gathered straight from the activation layout [batch][position]
// [channel] (im2col on the fly): forward  M = positions, N = out channels,
// K = 5 * in channels; input gradient M = positions, N = in channels,
// K = 5 * out channels; weight gradient M = 5 * in channels, N = out
// channels, K = positions (split over blocks, reduced with atomics).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sd.h"
#include "sd_internal.h"

namespace {

constexpr int PF = SD_PRED_FEATURES;  // input channels
constexpr int PC = 128;               // hidden channels
constexpr int PB = SD_PRED_BANDS;     // output channels
constexpr int PK = 5;                 // taps
constexpr int NLAYER = 4;
constexpr int CIN[NLAYER] = {PF, PC, PC, PC};
constexpr int COUT[NLAYER] = {PC, PC, PC, PB};

constexpr int64_t wcount(int l) { return (int64_t)PK * CIN[l] * COUT[l]; }
constexpr int64_t pcount(int l) { return wcount(l) + COUT[l]; }
constexpr int64_t NPARAM = pcount(0) + pcount(1) + pcount(2) + pcount(3);

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Warp-tile GEMM core: one warp accumulates a 16 x (8*NT) tile of
// C = A * B over k in [k0, k1) (k1 - k0 a multiple of 16 after padding; the
// operand getters return 0 outside the matrix).
template <int NT, class GA, class GB>
__device__ __forceinline__ void warp_gemm(int m0, int n0, int k0, int k1, const GA &ga,
                                          const GB &gb, float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  for (int k = k0; k < k1; k += 16) {
    uint32_t a[4];
    const int ka = k + q * 2;
    a[0] = pack2(ga(m0 + g, ka), ga(m0 + g, ka + 1));
    a[1] = pack2(ga(m0 + g + 8, ka), ga(m0 + g + 8, ka + 1));
    a[2] = pack2(ga(m0 + g, ka + 8), ga(m0 + g, ka + 9));
    a[3] = pack2(ga(m0 + g + 8, ka + 8), ga(m0 + g + 8, ka + 9));
#pragma unroll
    for (int j = 0; j < NT; j++) {
      const int n = n0 + j * 8 + g;
      const uint32_t b0 = pack2(gb(ka, n), gb(ka + 1, n));
      const uint32_t b1 = pack2(gb(ka + 8, n), gb(ka + 9, n));
      mma16816(acc[j], a, b0, b1);
    }
  }
}

struct Shape {
  int B, L;
  const int *len;  // device, B lengths
};

// ---- forward: z = conv(x) + b; h = relu(z) (hidden) or y = z (last) ----
template <int NT>
__global__ void __launch_bounds__(128) k_conv_fwd(Shape S, const __nv_bfloat16 *__restrict__ x,
                                                  int cin, const __nv_bfloat16 *__restrict__ W,
                                                  const float *__restrict__ bias, int cout,
                                                  int relu, __nv_bfloat16 *hout, float *yout) {
  const int M = S.B * S.L, K = PK * cin;
  const int m0 = (blockIdx.x * 4 + (threadIdx.x >> 5)) * 16, n0 = blockIdx.y * 8 * NT;
  auto ga = [&](int m, int k) -> float {
    if (m >= M || k >= K) return 0.f;
    const int b = m / S.L, l = m % S.L, t = k / cin, ci = k % cin;
    const int pos = l + t - 2;
    if (pos < 0 || pos >= __ldg(&S.len[b])) return 0.f;
    return __bfloat162float(x[((int64_t)b * S.L + pos) * cin + ci]);
  };
  auto gb = [&](int k, int n) -> float {
    if (k >= K || n >= cout) return 0.f;
    return __bfloat162float(W[(int64_t)k * cout + n]);
  };
  float acc[NT][4] = {};
  warp_gemm<NT>(m0, n0, 0, K, ga, gb, acc);
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; j++)
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int m = m0 + g + (r >= 2 ? 8 : 0), n = n0 + j * 8 + q * 2 + (r & 1);
      if (m >= M || n >= cout) continue;
      const int b = m / S.L, l = m % S.L;
      float v = acc[j][r] + bias[n];
      if (l >= __ldg(&S.len[b])) v = 0.f;
      if (relu) v = fmaxf(v, 0.f);
      if (hout) hout[(int64_t)m * cout + n] = __float2bfloat16_rn(v);
      if (yout) yout[(int64_t)m * cout + n] = v;
    }
}

// ---- input gradient: dzprev = (W^T conv dz) * [hprev > 0] ----
template <int NT>
__global__ void __launch_bounds__(128) k_conv_dgrad(Shape S, const float *__restrict__ dz, int cout,
                                                    const __nv_bfloat16 *__restrict__ W, int cin,
                                                    const __nv_bfloat16 *__restrict__ hprev,
                                                    float *dzprev) {
  const int M = S.B * S.L, K = PK * cout;
  const int m0 = (blockIdx.x * 4 + (threadIdx.x >> 5)) * 16, n0 = blockIdx.y * 8 * NT;
  auto ga = [&](int m, int k) -> float {
    if (m >= M || k >= K) return 0.f;
    const int b = m / S.L, l = m % S.L, t = k / cout, co = k % cout;
    const int pos = l - t + 2;
    if (pos < 0 || pos >= __ldg(&S.len[b])) return 0.f;
    return dz[((int64_t)b * S.L + pos) * cout + co];
  };
  auto gb = [&](int k, int n) -> float {
    if (k >= K || n >= cin) return 0.f;
    const int t = k / cout, co = k % cout;
    return __bfloat162float(W[((int64_t)t * cin + n) * cout + co]);
  };
  float acc[NT][4] = {};
  warp_gemm<NT>(m0, n0, 0, (K + 15) & ~15, ga, gb, acc);
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; j++)
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int m = m0 + g + (r >= 2 ? 8 : 0), n = n0 + j * 8 + q * 2 + (r & 1);
      if (m >= M || n >= cin) continue;
      const int b = m / S.L, l = m % S.L;
      float v = acc[j][r];
      if (l >= __ldg(&S.len[b]) || !(__bfloat162float(hprev[(int64_t)m * cin + n]) > 0.f)) v = 0.f;
      dzprev[(int64_t)m * cin + n] = v;
    }
}

// ---- weight gradient: dW[t*cin+ci][co] += sum over positions of x * dz ----
template <int NT>
__global__ void __launch_bounds__(128) k_conv_wgrad(Shape S, const __nv_bfloat16 *__restrict__ x,
                                                    int cin, const float *__restrict__ dz, int cout,
                                                    float *dW, int kchunk) {
  const int R = PK * cin, M = S.B * S.L;
  const int r0 = (blockIdx.x * 4 + (threadIdx.x >> 5)) * 16, n0 = blockIdx.y * 8 * NT;
  const int k0 = blockIdx.z * kchunk, k1 = min(M, k0 + kchunk);
  auto ga = [&](int r, int m) -> float {
    if (r >= R || m >= k1 || m >= M) return 0.f;
    const int t = r / cin, ci = r % cin, b = m / S.L, l = m % S.L;
    const int pos = l + t - 2, len = __ldg(&S.len[b]);
    if (l >= len || pos < 0 || pos >= len) return 0.f;
    return __bfloat162float(x[((int64_t)b * S.L + pos) * cin + ci]);
  };
  auto gb = [&](int m, int n) -> float {
    if (m >= k1 || m >= M || n >= cout) return 0.f;
    return dz[(int64_t)m * cout + n];
  };
  float acc[NT][4] = {};
  warp_gemm<NT>(r0, n0, k0, k0 + ((k1 - k0 + 15) & ~15), ga, gb, acc);
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; j++)
#pragma unroll
    for (int rr = 0; rr < 4; rr++) {
      const int r = r0 + g + (rr >= 2 ? 8 : 0), n = n0 + j * 8 + q * 2 + (rr & 1);
      if (r < R && n < cout && acc[j][rr] != 0.f) atomicAdd(&dW[(int64_t)r * cout + n], acc[j][rr]);
    }
}

__global__ void k_bias_grad(Shape S, const float *__restrict__ dz, int cout, float *db) {
  const int M = S.B * S.L;
  for (int n = threadIdx.x; n < cout; n += blockDim.x) {
    float s = 0.f;
    for (int m = blockIdx.x; m < M; m += gridDim.x) s += dz[(int64_t)m * cout + n];
    atomicAdd(&db[n], s);
  }
}

// mean squared error over the valid (position, band) entries
__global__ void k_mse(Shape S, const float *__restrict__ y, const float *__restrict__ target,
                      float inv_count, float *dz, float *loss) {
  const int M = S.B * S.L;
  float part = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * PB; e += gridDim.x * blockDim.x) {
    const int m = e / PB, b = m / S.L, l = m % S.L;
    float d = 0.f;
    if (l < __ldg(&S.len[b])) {
      const float r = y[e] - target[e];
      part += r * r;
      d = 2.f * r * inv_count;
    }
    dz[e] = d;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part * inv_count);
}

__global__ void k_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_to_bf16(int64_t n, const float *src, __nv_bfloat16 *dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(1024, (n + 255) / 256); }

}  // namespace

// ---------------------------------------------------------------------------
// host object
// ---------------------------------------------------------------------------
struct sd_predictor {
  float *w = nullptr;           // FP32 master parameters (all layers), device
  float *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr;  // BF16 copy of the parameters used by the kernels
  int64_t step = 0;
  // workspace for the current batch shape
  int cap_m = 0;
  __nv_bfloat16 *act[NLAYER] = {};  // layer inputs: act[0] features, act[l] = h_{l-1}
  float *y = nullptr, *tgt = nullptr, *loss = nullptr;  // loss: device scalar
  float *dz[NLAYER] = {};           // gradient of each layer's pre-activation
  int *len = nullptr;
};

namespace {

int64_t poff(int l) {
  int64_t o = 0;
  for (int q = 0; q < l; q++) o += pcount(q);
  return o;
}

template <class T>
bool dalloc(T *&p, int64_t count) {
  if (p) cudaFree(p);
  p = nullptr;
  return cudaMalloc(&p, sizeof(T) * (count > 0 ? count : 1)) == cudaSuccess;
}

int ensure(sd_predictor *P, int B, int L) {
  const int M = B * L;
  if (M <= P->cap_m) return SD_OK;
  const int cap = M + M / 2 + 64;
  bool ok = true;
  for (int l = 0; l < NLAYER; l++) ok = ok && dalloc(P->act[l], (int64_t)cap * CIN[l]);
  for (int l = 0; l < NLAYER; l++) ok = ok && dalloc(P->dz[l], (int64_t)cap * COUT[l]);
  ok = ok && dalloc(P->y, (int64_t)cap * PB) && dalloc(P->tgt, (int64_t)cap * PB) &&
       dalloc(P->len, cap);
  if (!ok) return SD_ENOMEM;
  P->cap_m = cap;
  return SD_OK;
}

void sync_bf16(sd_predictor *P) { k_to_bf16<<<grid_for(NPARAM), 256>>>(NPARAM, P->w, P->wb); }

template <int NT>
void fwd_layer(sd_predictor *P, Shape S, int l, __nv_bfloat16 *hout, float *yout) {
  const int M = S.B * S.L;
  dim3 grid((M + 63) / 64, (COUT[l] + 8 * NT - 1) / (8 * NT));
  const __nv_bfloat16 *W = P->wb + poff(l);
  const float *bias = P->w + poff(l) + wcount(l);
  k_conv_fwd<NT><<<grid, 128>>>(S, P->act[l], CIN[l], W, bias, COUT[l], l < NLAYER - 1, hout,
                                yout);
}

int forward(sd_predictor *P, int B, int L, const float *feats, const int *lengths, Shape &S) {
  if ((int64_t)B * L > (1 << 26)) return SD_EINVAL;
  for (int b = 0; b < B; b++)
    if (lengths[b] < 0 || lengths[b] > L) return SD_EINVAL;
  int rc = ensure(P, B, L);
  if (rc != SD_OK) return rc;
  const int M = B * L;
  std::vector<__nv_bfloat16> xb((size_t)M * PF);
  for (size_t k = 0; k < xb.size(); k++) xb[k] = __float2bfloat16_rn(feats[k]);
  if (cudaMemcpy(P->act[0], xb.data(), xb.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(P->len, lengths, sizeof(int) * B, cudaMemcpyHostToDevice) != cudaSuccess)
    return SD_ECUDA;
  S = Shape{B, L, P->len};
  for (int l = 0; l < NLAYER - 1; l++) fwd_layer<4>(P, S, l, P->act[l + 1], nullptr);
  fwd_layer<1>(P, S, NLAYER - 1, nullptr, P->y);
  return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

// gradients of the mean squared error into P->g (zeroed first); loss to *loss
int backward(sd_predictor *P, int B, int L, const float *feats, const float *targets,
             const int *lengths, float *loss) {
  Shape S;
  int rc = forward(P, B, L, feats, lengths, S);
  if (rc != SD_OK) return rc;
  const int M = B * L;
  int64_t valid = 0;
  for (int b = 0; b < B; b++) valid += std::max(0, std::min(lengths[b], L));
  const float inv = valid > 0 ? 1.f / (float)(valid * PB) : 0.f;
  if (cudaMemcpy(P->tgt, targets, sizeof(float) * M * PB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(P->loss, 0, sizeof(float)) != cudaSuccess ||
      cudaMemset(P->g, 0, sizeof(float) * NPARAM) != cudaSuccess)
    return SD_ECUDA;
  k_mse<<<grid_for((int64_t)M * PB), 256>>>(S, P->y, P->tgt, inv, P->dz[NLAYER - 1], P->loss);
  for (int l = NLAYER - 1; l >= 0; l--) {
    float *dW = P->g + poff(l), *db = dW + wcount(l);
    const int R = PK * CIN[l];
    const int kchunk = 2048;
    dim3 gw((R + 63) / 64, (COUT[l] + 31) / 32, (M + kchunk - 1) / kchunk);
    if (COUT[l] >= 32) {
      k_conv_wgrad<4><<<gw, 128>>>(S, P->act[l], CIN[l], P->dz[l], COUT[l], dW, kchunk);
    } else {
      dim3 gw1((R + 63) / 64, (COUT[l] + 7) / 8, (M + kchunk - 1) / kchunk);
      k_conv_wgrad<1><<<gw1, 128>>>(S, P->act[l], CIN[l], P->dz[l], COUT[l], dW, kchunk);
    }
    k_bias_grad<<<64, 128>>>(S, P->dz[l], COUT[l], db);
    if (l > 0) {
      dim3 gd((M + 63) / 64, (CIN[l] + 31) / 32);
      k_conv_dgrad<4><<<gd, 128>>>(S, P->dz[l], COUT[l], P->wb + poff(l), CIN[l], P->act[l],
                                   P->dz[l - 1]);
    }
  }
  if (cudaMemcpy(loss, P->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SD_ECUDA;
  return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

// deterministic parameter initialisation (splitmix64 stream, He-uniform)
uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" int64_t sd_pred_num_params(void) { return NPARAM; }

extern "C" int sd_pred_create(uint64_t seed, sd_predictor **out) {
  if (!out) return SD_EINVAL;
  *out = nullptr;
  sd_predictor *P = new (std::nothrow) sd_predictor();
  if (!P) return SD_ENOMEM;
  std::vector<float> h(NPARAM, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < NLAYER; l++) {
    const float bound = std::sqrt(6.f / (float)(PK * CIN[l]));
    float *W = h.data() + poff(l);
    for (int64_t k = 0; k < wcount(l); k++) {
      const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      W[k] = (float)((2.0 * u - 1.0) * bound);
    }
  }
  bool ok = dalloc(P->w, NPARAM) && dalloc(P->g, NPARAM) && dalloc(P->m, NPARAM) &&
            dalloc(P->v, NPARAM) && dalloc(P->wb, NPARAM) && dalloc(P->loss, 1);
  ok = ok && cudaMemcpy(P->w, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(P->m, 0, sizeof(float) * NPARAM) == cudaSuccess &&
       cudaMemset(P->v, 0, sizeof(float) * NPARAM) == cudaSuccess;
  if (!ok) {
    sd_pred_free(P);
    return SD_ECUDA;
  }
  sync_bf16(P);
  *out = P;
  return SD_OK;
}

extern "C" void sd_pred_free(sd_predictor *P) {
  if (!P) return;
  cudaFree(P->w);
  cudaFree(P->g);
  cudaFree(P->m);
  cudaFree(P->v);
  cudaFree(P->wb);
  cudaFree(P->loss);
  for (int l = 0; l < NLAYER; l++) {
    cudaFree(P->act[l]);
    cudaFree(P->dz[l]);
  }
  cudaFree(P->y);
  cudaFree(P->tgt);
  cudaFree(P->len);
  delete P;
}

extern "C" int sd_pred_get_params(const sd_predictor *P, float *params) {
  if (!P || !params) return SD_EINVAL;
  return cudaMemcpy(params, P->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess
             ? SD_OK
             : SD_ECUDA;
}

extern "C" int sd_pred_set_params(sd_predictor *P, const float *params) {
  if (!P || !params) return SD_EINVAL;
  if (cudaMemcpy(P->w, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
    return SD_ECUDA;
  sync_bf16(P);
  P->step = 0;
  cudaMemset(P->m, 0, sizeof(float) * NPARAM);
  cudaMemset(P->v, 0, sizeof(float) * NPARAM);
  return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

extern "C" int sd_pred_forward(sd_predictor *P, int B, int L, const float *feats,
                               const int *lengths, float *out) {
  if (!P || B <= 0 || L <= 0 || !feats || !lengths || !out) return SD_EINVAL;
  Shape S;
  int rc = forward(P, B, L, feats, lengths, S);
  if (rc != SD_OK) return rc;
  return cudaMemcpy(out, P->y, sizeof(float) * B * L * PB, cudaMemcpyDeviceToHost) == cudaSuccess
             ? SD_OK
             : SD_ECUDA;
}

extern "C" int sd_pred_gradients(sd_predictor *P, int B, int L, const float *feats,
                                 const float *targets, const int *lengths, float *grads,
                                 float *loss) {
  if (!P || B <= 0 || L <= 0 || !feats || !targets || !lengths || !loss) return SD_EINVAL;
  int rc = backward(P, B, L, feats, targets, lengths, loss);
  if (rc != SD_OK) return rc;
  if (grads && cudaMemcpy(grads, P->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SD_ECUDA;
  return SD_OK;
}

extern "C" int sd_pred_train_step(sd_predictor *P, int B, int L, const float *feats,
                                  const float *targets, const int *lengths, float lr,
                                  float *loss) {
  if (!P || !(lr > 0.f)) return SD_EINVAL;
  int rc = sd_pred_gradients(P, B, L, feats, targets, lengths, nullptr, loss);
  if (rc != SD_OK) return rc;
  P->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)P->step), c2 = 1.f - std::pow(b2, (float)P->step);
  k_adam<<<grid_for(NPARAM), 256>>>(NPARAM, P->w, P->g, P->m, P->v, lr, b1, b2, 1e-8f, c1, c2);
  sync_bf16(P);
  return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

// Input features of one protein: per codon position, 32 floats:
// [0,21) one-hot amino acid (ACDEFGHIKLMNPQRSTVWY, then '*'), [21,27) the
// weights of its synonymous codons in decreasing order (0 padded),
// 27 lambda/4, 28 ln(A)/8, 29 position / A, 30-31 zero.
extern "C" int sd_pred_features(const char *protein, const double *w, double lambda, float *feat) {
  if (!protein || !w || !feat || !(lambda >= 0.0)) return SD_EINVAL;
  static const char *aas = "ACDEFGHIKLMNPQRSTVWY*";
  const int A = (int)std::strlen(protein);
  for (int k = 0; k < A; k++) {
    float *f = feat + (size_t)k * PF;
    for (int c = 0; c < PF; c++) f[c] = 0.f;
    const char *hit = std::strchr(aas, protein[k]);
    if (!hit || !*hit) return SD_EINVAL;
    f[hit - aas] = 1.f;
    double ws[6];
    int nw = 0;
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++)
          if (sd_internal_translate(x, y, z) == protein[k] && nw < 6) ws[nw++] = w[16 * x + 4 * y + z];
    for (int a = 0; a < nw; a++)
      for (int b = a + 1; b < nw; b++)
        if (ws[b] > ws[a]) std::swap(ws[a], ws[b]);
    for (int a = 0; a < nw; a++) f[21 + a] = (float)ws[a];
    f[27] = (float)(lambda / 4.0);
    f[28] = (float)(std::log((double)A) / 8.0);
    f[29] = (float)k / (float)A;
  }
  return SD_OK;
}
