// FP8 (E4M3) form of the frozen static predictor (the paper's static public model, §4.2.2, is
// frozen; the held-out configuration stores it in FP8).  One scale per channel, chosen so that the
// channel's largest magnitude maps to 448, the largest finite E4M3 value:
//   embedding table   one scale for the whole table
//   W1 (stored W1t)   one scale per hidden unit (a row of W1t)
//   W2                one scale per logit (a column of W2), codes stored transposed [A][H] so the
//                     logits GEMM reads them K-major
// scale = amax / 448 (an all-zero channel has scale 1), code = E4M3(w / scale) rounded to nearest
// even with saturation, both divisions correctly rounded FP32.  The channel maximum is an
// order-free reduction, so the codes do not depend on scheduling.
#include <cuda_fp8.h>

#include "internal.h"

namespace pmklc {

namespace {

constexpr int kQThreads = 256;

__device__ __forceinline__ uint8_t e4m3(float x) {
  return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Block b quantises channel b: n elements src[b * ch_stride + i * el_stride] into dst[b * n + i].
__global__ void __launch_bounds__(kQThreads) quant_channels_kernel(const float *__restrict__ src, int n,
                                                                   size_t ch_stride, size_t el_stride,
                                                                   uint8_t *__restrict__ dst,
                                                                   float *__restrict__ scale) {
  __shared__ float red[kQThreads / 32];
  const float *s = src + (size_t)blockIdx.x * ch_stride;
  float mx = 0.f;
  for (int i = threadIdx.x; i < n; i += kQThreads) mx = fmaxf(mx, fabsf(s[(size_t)i * el_stride]));
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.f;
  for (int w = 0; w < kQThreads / 32; ++w) mx = fmaxf(mx, red[w]);
  const float sc = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
  if (threadIdx.x == 0) scale[blockIdx.x] = sc;
  uint8_t *d = dst + (size_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += kQThreads) d[i] = e4m3(__fdiv_rn(s[(size_t)i * el_stride], sc));
}

// combined hidden-layer scale of each hidden unit: s_emb * s_w1[h] (FP32 product)
__global__ void fp8_hidden_scale_kernel(const float *scales, int H, float *c1) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < H) c1[h] = __fmul_rn(scales[0], scales[1 + h]);
}

}  // namespace

size_t fp8_code_bytes(const Dims &d) { return (size_t)d.A * d.E + (size_t)d.H * d.K1() + (size_t)d.A * d.H; }
size_t fp8_scale_count(const Dims &d) { return 1 + (size_t)d.H + (size_t)d.A; }

void launch_quantize_fp8(const float *d_params, const Dims &d, uint8_t *d_codes, float *d_scales, cudaStream_t st) {
  // embedding table: one channel of A*E elements
  quant_channels_kernel<<<1, kQThreads, 0, st>>>(d_params + d.off_emb(), d.A * d.E, 0, 1, d_codes, d_scales);
  // W1t: H channels (rows) of t*E elements
  quant_channels_kernel<<<d.H, kQThreads, 0, st>>>(d_params + d.off_w1(), d.K1(), (size_t)d.K1(), 1,
                                                   d_codes + (size_t)d.A * d.E, d_scales + 1);
  // W2 [H][A]: A channels (columns) of H elements, written transposed [A][H]
  quant_channels_kernel<<<d.A, kQThreads, 0, st>>>(d_params + d.off_w2(), d.H, 1, (size_t)d.A,
                                                   d_codes + (size_t)d.A * d.E + (size_t)d.H * d.K1(),
                                                   d_scales + 1 + d.H);
}

void launch_fp8_hidden_scale(const float *d_scales, const Dims &d, float *d_c1, cudaStream_t st) {
  fp8_hidden_scale_kernel<<<(d.H + 255) / 256, 256, 0, st>>>(d_scales, d.H, d_c1);
}

}  // namespace pmklc

using namespace pmklc;

extern "C" int pmklc_quantize_static_fp8(const float *d_params, uint32_t k, uint32_t E, uint32_t t, uint32_t H,
                                         uint8_t *d_codes, float *d_scales, void *stream) {
  if (k < 1 || k > 8 || !E || !t || !H || E > 4096 || t > 4096 || H > 65535 || !d_params || !d_codes || !d_scales)
    return PMKLC_EINVAL;
  const Dims d{1 << (2 * k), (int)E, (int)t, (int)H};
  cudaStream_t st = (cudaStream_t)stream;
  launch_quantize_fp8(d_params, d, d_codes, d_scales, st);
  PMKLC_CUDA_TRY(cudaGetLastError());
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  return PMKLC_OK;
}
