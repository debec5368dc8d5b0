// nn.h -- launchers of the surrogate's kernels (nn.cu), used by net.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gpe2p {
namespace nn {

// input normalisation and output map of the network:
//   network input  = (x[c] - mean[c]) * inv[c]                    (c < in channels)
//   network output = (residual ? x[c] : 0) + oscale[c] * head[c]  (c < out channels)
// and the loss is the mean of ((output - target) / oscale)^2
struct Norm {
  float mean[16], inv[16], oscale[16];
  int residual;
};

// one convolution (3x3 circular or 1x1) as implicit GEMMs; see nn.cu
struct ConvArgs {
  int B, H, W, npix;   // batch, height, width, B*H*W
  int cin, cout, taps; // channels in/out (multiples of 16), taps 9 (3x3) or 1 (1x1)
  // forward: y = act(z), z = conv(x) + bias
  const __nv_bfloat16* x;
  int ldx, xoff;       // x: row stride (channels per pixel) and channel offset
  int up;              // 1: x is stored at (H/2, W/2) and read as its nearest 2x upsampling
  const __nv_bfloat16* wt;  // [cout][taps*cin]
  const __nv_bfloat16* wtp; // the same packed per K chunk, [cin/16][9][2][cout][8] (tcgen05 forward)
  const float* bias;
  __nv_bfloat16* z;    // pre-activation [npix][cout] (or nullptr)
  __nv_bfloat16* y;
  int ldy, yoff, act;  // act: 1 SiLU, 0 identity
  // dgrad: dx (+)= conv^T(dz)
  const __nv_bfloat16* dz;  // [npix][cout]
  int ldz;
  const __nv_bfloat16* wd;  // [cin][taps*cout]
  const __nv_bfloat16* wdp; // the same packed per K chunk, [cout/16][9][2][cin][8] (tcgen05 data gradient)
  __nv_bfloat16* dx;
  int lddx, dxoff, accumulate;
  // wgrad: dw[co][tap*cin + ci] += sum over pixels (FP32, split over ksplit pixels per block)
  float* dw;
  int ksplit;
  int tc;     // 1: 3x3 forward and data gradient on the tcgen05 kernels (conv_tc.cu)
  int* err;   // device error word: set to 1 by a tcgen05 kernel whose wait timed out
  int wait_fault;  // test switch: the first wait of each tcgen05 CTA for a filled stage reports a timeout
};

cudaError_t conv_forward(const ConvArgs& a, cudaStream_t s);
// the tcgen05 forms (conv_tc.cu) and the shapes they take
bool conv_tc_supported(const ConvArgs& a, int mode);
cudaError_t conv_forward_tc(const ConvArgs& a, cudaStream_t s);
cudaError_t conv_dgrad_tc(const ConvArgs& a, cudaStream_t s);
cudaError_t conv_dgrad(const ConvArgs& a, cudaStream_t s);
cudaError_t conv_wgrad(const ConvArgs& a, cudaStream_t s);
// dZ = dY silu'(z) and db += sum over pixels of dZ
cudaError_t dsilu_bias(const __nv_bfloat16* dy, int ldy, int yoff, const __nv_bfloat16* z, __nv_bfloat16* dz,
                       long long npix, int c, float* db, cudaStream_t s);
cudaError_t pool_fwd(const __nv_bfloat16* x, int ldx, int xoff, __nv_bfloat16* y, int B, int H, int W, int c,
                     cudaStream_t s);
cudaError_t pool_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int ldx, int xoff, int B, int H, int W, int c,
                     int accumulate, cudaStream_t s);
cudaError_t up_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int B, int H, int W, int c, cudaStream_t s);
cudaError_t copy_ch(const __nv_bfloat16* src, int lds, int soff, __nv_bfloat16* dst, int ldd, int doff,
                    long long npix, int c, int accumulate, cudaStream_t s);
cudaError_t to_bf16(const float* x, int cin, __nv_bfloat16* y, int ldo, long long npix, const Norm& nm,
                    cudaStream_t s);
cudaError_t head_fwd(const __nv_bfloat16* x, int cin, const float* w, const float* b, float* y, int cout,
                     long long npix, const float* xin, int in_ch, const Norm& nm, cudaStream_t s);
cudaError_t head_bwd(const __nv_bfloat16* x, int cin, const float* w, const float* dy, int cout, __nv_bfloat16* dx,
                     float* dw, float* db, long long npix, cudaStream_t s);
cudaError_t mse(const float* y, const float* t, float* dy, long long n, int cout, const Norm& nm, float* loss,
                cudaStream_t s);
cudaError_t adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t s);
cudaError_t weights_bf16(const float* w, __nv_bfloat16* wt, __nv_bfloat16* wd, __nv_bfloat16* wtp,
                         __nv_bfloat16* wdp, int cout, int cin, int taps, cudaStream_t s);

}  // namespace nn
}  // namespace gpe2p
