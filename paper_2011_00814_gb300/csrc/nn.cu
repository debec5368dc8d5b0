// nn.cu -- kernels of the learned surrogate: a convolutional U-Net on the
// periodic 2D grid, BF16 activations and weights, FP32 accumulation on the
// tensor cores (mma.sync m16n8k16), FP32 master weights and Adam.
//
// Tensors are NHWC: element (b, y, x, c) of a tensor with row stride ldc
// (channels per pixel, >= the channels used) sits at ((b*H + y)*W + x)*ldc
// + coff + c.  Convolutions pad circularly (the domain is periodic).
//
// The three products of a 3x3 convolution are implicit GEMMs over
// k = tap*C + c (tap = 3*(dy+1) + (dx+1)):
//   forward  Z[p, co]   = sum_k X[p + off(tap), ci] WT[co][k]          (+ bias, SiLU)
//   dgrad    dX[p, ci]  = sum_k dZ[p - off(tap), co] WD[ci][tap*Cout + co]
//   wgrad    dWT[co][k] = sum_p dZ[p, co] X[p + off(tap), ci]          (split over p, FP32 atomics)
// with WT[co][tap*Cin + ci] the weights and WD[ci][tap*Cout + co] their
// transpose.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn.h"

namespace gpe2p {
namespace nn {

constexpr int BM = 64;
constexpr int BK = 32;
constexpr int NT = 128;       // 4 warps: 2 (m) x 2 (n)
constexpr int SKEW = 8;       // bf16 padding of a shared-memory row

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// pixel p of a batch -> (b, y, x)
__device__ __forceinline__ void pix(int p, int H, int W, int& b, int& y, int& x) {
  x = p % W;
  const int q = p / W;
  y = q % H;
  b = q / H;
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// ---------------------------------------------------------------------------
// implicit GEMM: forward (MODE 0), dgrad (MODE 1), wgrad (MODE 2)
// ---------------------------------------------------------------------------

template <int MODE, int BN>
__global__ void __launch_bounds__(NT) igemm_kernel(const ConvArgs a) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + SKEW];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + SKEW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;       // warp tile: 32 x BN/2
  constexpr int WN = BN / 2, NJ = WN / 8;         // n8 tiles per warp
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int ks = a.taps == 9 ? 9 : 1;

  float acc[2][NJ][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  // K range of this block
  int kbeg = 0, kend;
  if (MODE == 0) kend = ks * a.cin;
  else if (MODE == 1) kend = ks * a.cout;
  else {
    kbeg = blockIdx.z * a.ksplit;
    kend = min(kbeg + a.ksplit, a.npix);
  }

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // ---- stage the A and B tiles ----
    if (MODE != 2) {
      // A: BM rows (pixels) x BK (k); each thread 16 consecutive k of one row
      {
        const int r = tid >> 1, kk = k0 + (tid & 1) * 16;
        const int p = m0 + r;
        uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
        if (p < a.npix && kk < kend) {
          const int C = MODE == 0 ? a.cin : a.cout;
          const int tap = kk / C, c = kk - tap * C;
          int b, y, x;
          pix(p, a.H, a.W, b, y, x);
          int dy = 0, dx = 0;
          if (ks == 9) { dy = tap / 3 - 1; dx = tap % 3 - 1; }
          if (MODE == 1) { dy = -dy; dx = -dx; }
          int yy = wrapi(y + dy, a.H), xx = wrapi(x + dx, a.W);
          const __nv_bfloat16* src = MODE == 0 ? a.x : a.dz;
          const int ld = MODE == 0 ? a.ldx : a.ldz;
          const int off = MODE == 0 ? a.xoff : 0;
          int Hs = a.H, Ws = a.W;
          if (MODE == 0 && a.up) { yy >>= 1; xx >>= 1; Hs >>= 1; Ws >>= 1; }
          const uint4* s = reinterpret_cast<const uint4*>(src + ((size_t)(b * Hs + yy) * Ws + xx) * ld + off + c);
          v0 = s[0];
          v1 = s[1];
        }
        *reinterpret_cast<uint4*>(&As[r][(tid & 1) * 16]) = v0;
        *reinterpret_cast<uint4*>(&As[r][(tid & 1) * 16 + 8]) = v1;
      }
      // B: BN rows (output columns) x BK (k), from a k-contiguous weight copy
      for (int q = tid; q < BN * 2; q += NT) {
        const int r = q >> 1, kk = k0 + (q & 1) * 16;
        const int n = n0 + r;
        uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
        const int N = MODE == 0 ? a.cout : a.cin;
        if (n < N && kk < kend) {
          const __nv_bfloat16* w = MODE == 0 ? a.wt : a.wd;
          const int K = MODE == 0 ? ks * a.cin : ks * a.cout;
          const uint4* s = reinterpret_cast<const uint4*>(w + (size_t)n * K + kk);
          v0 = s[0];
          v1 = s[1];
        }
        *reinterpret_cast<uint4*>(&Bs[r][(q & 1) * 16]) = v0;
        *reinterpret_cast<uint4*>(&Bs[r][(q & 1) * 16 + 8]) = v1;
      }
    } else {
      // wgrad: A = dZ^T (rows co, k = pixel), B = X-gather^T (rows (tap, ci), k = pixel);
      // each thread reads 8 channels of one pixel and scatters them into a column
      for (int q = tid; q < BK * (BM / 8); q += NT) {
        const int pl = q / (BM / 8), cg = (q % (BM / 8)) * 8;
        const int p = k0 + pl, co = m0 + cg;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (p < kend && co < a.cout)
          v = *reinterpret_cast<const uint4*>(a.dz + (size_t)p * a.ldz + co);
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) As[cg + j][pl] = e[j];
      }
      for (int q = tid; q < BK * (BN / 8); q += NT) {
        const int pl = q / (BN / 8), ng = (q % (BN / 8)) * 8;
        const int p = k0 + pl, n = n0 + ng;   // n = tap*cin + ci
        uint4 v = make_uint4(0, 0, 0, 0);
        if (p < kend && n < ks * a.cin) {
          const int tap = n / a.cin, ci = n - tap * a.cin;
          int b, y, x;
          pix(p, a.H, a.W, b, y, x);
          int dy = 0, dx = 0;
          if (ks == 9) { dy = tap / 3 - 1; dx = tap % 3 - 1; }
          int yy = wrapi(y + dy, a.H), xx = wrapi(x + dx, a.W);
          int Hs = a.H, Ws = a.W;
          if (a.up) { yy >>= 1; xx >>= 1; Hs >>= 1; Ws >>= 1; }
          v = *reinterpret_cast<const uint4*>(a.x + ((size_t)(b * Hs + yy) * Ws + xx) * a.ldx + a.xoff + ci);
        }
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) Bs[ng + j][pl] = e[j];
      }
    }
    __syncthreads();
    // ---- two k16 steps of mma ----
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4], bf[NJ][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r + g][kk + 2 * t]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + g + 8][kk + 2 * t]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r + g][kk + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + g + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int c = wn * WN + j * 8;
        bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c + g][kk + 2 * t]);
        bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c + g][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }

  // ---- epilogue ----
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 32 + i * 16 + g + h * 8;
        const int n = n0 + wn * WN + j * 8 + 2 * t;
        const float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (MODE == 0) {
          if (m < a.npix && n < a.cout) {
            const float z0 = v0 + a.bias[n], z1 = v1 + a.bias[n + 1];
            if (a.z) {
              __nv_bfloat162 zz = __floats2bfloat162_rn(z0, z1);
              *reinterpret_cast<__nv_bfloat162*>(a.z + (size_t)m * a.cout + n) = zz;
            }
            const float y0 = a.act ? silu(z0) : z0, y1 = a.act ? silu(z1) : z1;
            *reinterpret_cast<__nv_bfloat162*>(a.y + (size_t)m * a.ldy + a.yoff + n) = __floats2bfloat162_rn(y0, y1);
          }
        } else if (MODE == 1) {
          if (m < a.npix && n < a.cin) {
            __nv_bfloat16* dst = a.dx + (size_t)m * a.lddx + a.dxoff + n;
            float d0 = v0, d1 = v1;
            if (a.accumulate) {
              d0 += __bfloat162float(dst[0]);
              d1 += __bfloat162float(dst[1]);
            }
            *reinterpret_cast<__nv_bfloat162*>(dst) = __floats2bfloat162_rn(d0, d1);
          }
        } else {
          if (m < a.cout && n < ks * a.cin) {
            atomicAdd(a.dw + (size_t)m * ks * a.cin + n, v0);
            atomicAdd(a.dw + (size_t)m * ks * a.cin + n + 1, v1);
          }
        }
      }
}

// ---------------------------------------------------------------------------
// element-wise and small kernels
// ---------------------------------------------------------------------------

static unsigned blocks_for(long long n, int per = 256) {
  long long b = (n + per - 1) / per;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)(b < 1 ? 1 : b);
}

// eight BF16 channels <-> floats
__device__ __forceinline__ void unpack8(const uint4& v, float f[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 t = __bfloat1622float2(h[e]);
    f[2 * e] = t.x;
    f[2 * e + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float f[8]) {
  uint4 v;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
  for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
  return v;
}
__device__ __forceinline__ uint4 ld8(const __nv_bfloat16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st8(__nv_bfloat16* p, const uint4& v) { *reinterpret_cast<uint4*>(p) = v; }

// dZ = dY * silu'(z) (dY read with row stride ldy and channel offset yoff) and
// db[c] += sum over pixels of the stored dZ; a thread takes 8 channels of a pixel
__global__ void dsilu_bias_kernel(const __nv_bfloat16* dy, int ldy, int yoff, const __nv_bfloat16* z,
                                  __nv_bfloat16* dz, long long npix, int c, float* db) {
  extern __shared__ float red[];  // c
  const int G = c >> 3, lanes = blockDim.x / G;
  const int g = threadIdx.x % G, pl = threadIdx.x / G;
  for (int q = threadIdx.x; q < c; q += blockDim.x) red[q] = 0.f;
  __syncthreads();
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long long p = blockIdx.x * (long long)lanes + pl; p < npix; p += (long long)gridDim.x * lanes) {
    float gy[8], zz[8], d[8];
    unpack8(ld8(dy + p * ldy + yoff + 8 * g), gy);
    unpack8(ld8(z + p * c + 8 * g), zz);
#pragma unroll
    for (int e = 0; e < 8; ++e) d[e] = gy[e] * dsilu(zz[e]);
    const uint4 o = pack8(d);
    st8(dz + p * c + 8 * g, o);
    float r[8];
    unpack8(o, r);
#pragma unroll
    for (int e = 0; e < 8; ++e) s[e] += r[e];
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) atomicAdd(&red[8 * g + e], s[e]);
  __syncthreads();
  for (int q = threadIdx.x; q < c; q += blockDim.x) atomicAdd(db + q, red[q]);
}

// 2x2 average pooling (forward) and its adjoint; a thread takes 8 channels
__global__ void pool_fwd_kernel(const __nv_bfloat16* x, int ldx, int xoff, __nv_bfloat16* y, int B, int H, int W,
                                int c) {
  const int Ho = H / 2, Wo = W / 2, G = c >> 3;
  const long long n = (long long)B * Ho * Wo * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % G);
    long long q = i / G;
    const int xo = (int)(q % Wo);
    const long long r = q / Wo;
    const int yo = (int)(r % Ho);
    const int b = (int)(r / Ho);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, f[8];
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        unpack8(ld8(x + ((size_t)(b * H + 2 * yo + dy) * W + 2 * xo + dx) * ldx + xoff + 8 * g), f);
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] += f[e];
      }
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] *= 0.25f;
    st8(y + q * c + 8 * g, pack8(acc));
  }
}

// dX (row stride ldx, offset xoff) = 1/4 dY spread; accumulate adds to dX
__global__ void pool_bwd_kernel(const __nv_bfloat16* dy, __nv_bfloat16* dx, int ldx, int xoff, int B, int H, int W,
                                int c, int accumulate) {
  const int G = c >> 3;
  const long long n = (long long)B * H * W * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % G);
    const long long q = i / G;
    const int x = (int)(q % W);
    const long long r = q / W;
    const int y = (int)(r % H);
    const int b = (int)(r / H);
    float f[8];
    unpack8(ld8(dy + ((size_t)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * c + 8 * g), f);
    __nv_bfloat16* d = dx + q * ldx + xoff + 8 * g;
    float o[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (accumulate) unpack8(ld8(d), o);
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] += 0.25f * f[e];
    st8(d, pack8(o));
  }
}

// adjoint of the nearest 2x upsampling: the sum of the four children
__global__ void up_bwd_kernel(const __nv_bfloat16* dy, __nv_bfloat16* dx, int B, int H, int W, int c) {
  const int Hi = H / 2, Wi = W / 2, G = c >> 3;  // H, W of dY
  const long long n = (long long)B * Hi * Wi * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % G);
    const long long q = i / G;
    const int xo = (int)(q % Wi);
    const long long r = q / Wi;
    const int yo = (int)(r % Hi);
    const int b = (int)(r / Hi);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, f[8];
    for (int dy2 = 0; dy2 < 2; ++dy2)
      for (int dx2 = 0; dx2 < 2; ++dx2) {
        unpack8(ld8(dy + ((size_t)(b * H + 2 * yo + dy2) * W + 2 * xo + dx2) * c + 8 * g), f);
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] += f[e];
      }
    st8(dx + q * c + 8 * g, pack8(acc));
  }
}

// copy c channels from (src, lds, soff) to (dst, ldd, doff); accumulate adds
__global__ void copy_ch_kernel(const __nv_bfloat16* src, int lds, int soff, __nv_bfloat16* dst, int ldd, int doff,
                               long long npix, int c, int accumulate) {
  const int G = c >> 3;
  const long long n = npix * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / G;
    const int g = (int)(i - p * G);
    const uint4 v = ld8(src + p * lds + soff + 8 * g);
    __nv_bfloat16* d = dst + p * ldd + doff + 8 * g;
    if (accumulate) {
      float a[8], b[8];
      unpack8(v, a);
      unpack8(ld8(d), b);
#pragma unroll
      for (int e = 0; e < 8; ++e) a[e] += b[e];
      st8(d, pack8(a));
    } else {
      st8(d, v);
    }
  }
}

// FP32 NHWC (cin channels) -> normalised BF16 NHWC padded to ldo channels with zeros
__global__ void to_bf16_kernel(const float* x, int cin, __nv_bfloat16* y, int ldo, long long npix, const Norm nm) {
  const long long n = npix * ldo;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / ldo;
    const int ch = (int)(i - p * ldo);
    y[i] = __float2bfloat16_rn(ch < cin ? (x[p * cin + ch] - nm.mean[ch]) * nm.inv[ch] : 0.f);
  }
}

// the same for the network's input row of 16 channels (cin <= 16): a thread
// takes a pixel, reads its cin values once and writes its 16 BF16 channels
// as two 16-byte stores
__global__ void to_bf16_16_kernel(const float* x, int cin, __nv_bfloat16* y, long long npix, const Norm nm) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    uint4 o[2];
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(o);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c0 = 2 * e, c1 = 2 * e + 1;
      const float v0 = c0 < cin ? (x[p * cin + c0] - nm.mean[c0]) * nm.inv[c0] : 0.f;
      const float v1 = c1 < cin ? (x[p * cin + c1] - nm.mean[c1]) * nm.inv[c1] : 0.f;
      h[e] = __halves2bfloat162(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
    }
    uint4* dst = reinterpret_cast<uint4*>(y + p * 16);
    dst[0] = o[0];
    dst[1] = o[1];
  }
}

// output layer: 1x1 convolution cin -> cout (cout <= 16), FP32 out, no activation, then the
// output map (scale, optional residual from the raw FP32 input xin of in_ch channels);
// a thread takes one pixel, weights in shared memory
__global__ void head_fwd_kernel(const __nv_bfloat16* x, int cin, const float* w, const float* b, float* y, int cout,
                                long long npix, const float* xin, int in_ch, const Norm nm) {
  extern __shared__ __align__(16) float sw[];  // [cout][cin], bias[cout]
  for (int q = threadIdx.x; q < cout * cin + cout; q += blockDim.x) sw[q] = q < cout * cin ? w[q] : b[q - cout * cin];
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    float acc[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) acc[o] = o < cout ? sw[cout * cin + o] : 0.f;
    for (int c0 = 0; c0 < cin; c0 += 8) {
      float f[8];
      unpack8(ld8(x + p * cin + c0), f);
#pragma unroll
      for (int o = 0; o < 16; ++o) {
        if (o < cout) {
          const float* wr = sw + o * cin + c0;
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[o] += wr[e] * f[e];
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 16; ++o)
      if (o < cout) y[p * cout + o] = (nm.residual ? xin[p * in_ch + o] : 0.f) + nm.oscale[o] * acc[o];
  }
}

// its adjoint: dX = dY W (bf16), dW += sum_p dY x^T, db += sum_p dY.  A block stages a tile
// of TP pixels; thread t computes dX of pixel t, and each (o, c) pair of dW, db is
// accumulated by one thread in shared memory.
__global__ void head_bwd_kernel(const __nv_bfloat16* x, int cin, const float* w, const float* dy, int cout,
                                __nv_bfloat16* dx, float* dw, float* db, long long npix, int TP) {
  extern __shared__ __align__(16) float sh[];
  const int npair = cout * cin + cout;
  float* sacc = sh;                         // npair
  float* sw = sacc + npair;                 // cout * cin
  float* sdy = sw + cout * cin;             // TP * cout
  // the staged activations start on a 16-byte boundary (they are moved 8 channels at a time)
  const int nf = (npair + cout * cin + TP * cout + 3) & ~3;
  __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(sh + nf);   // TP * cin
  for (int q = threadIdx.x; q < npair; q += blockDim.x) sacc[q] = 0.f;
  for (int q = threadIdx.x; q < cout * cin; q += blockDim.x) sw[q] = w[q];
  for (long long p0 = (long long)blockIdx.x * TP; p0 < npix; p0 += (long long)gridDim.x * TP) {
    const int np = (int)(npix - p0 < TP ? npix - p0 : TP);
    __syncthreads();
    for (int q = threadIdx.x; q < np * cout; q += blockDim.x) sdy[q] = dy[p0 * cout + q];
    for (int q = threadIdx.x; q < np * (cin >> 3); q += blockDim.x)
      st8(sx + q * 8, ld8(x + p0 * cin + (long long)q * 8));
    __syncthreads();
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
      for (int c0 = 0; c0 < cin; c0 += 8) {
        float d[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int o = 0; o < cout; ++o) {
          const float g = sdy[t * cout + o];
#pragma unroll
          for (int e = 0; e < 8; ++e) d[e] += g * sw[o * cin + c0 + e];
        }
        st8(dx + (p0 + t) * cin + c0, pack8(d));
      }
    }
    for (int q = threadIdx.x; q < npair; q += blockDim.x) {
      float acc = 0.f;
      if (q < cout * cin) {
        const int o = q / cin, c = q - o * cin;
        for (int t = 0; t < np; ++t) acc += sdy[t * cout + o] * __bfloat162float(sx[t * cin + c]);
      } else {
        const int o = q - cout * cin;
        for (int t = 0; t < np; ++t) acc += sdy[t * cout + o];
      }
      sacc[q] += acc;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < cout * cin; q += blockDim.x) atomicAdd(dw + q, sacc[q]);
  for (int q = threadIdx.x; q < cout; q += blockDim.x) atomicAdd(db + q, sacc[cout * cin + q]);
}

// mean squared error of the scaled output error e = (y - t) / oscale and its gradient with
// respect to the head's output: loss += sum e^2 / n, dy = 2 e / n
__global__ void mse_kernel(const float* y, const float* t, float* dy, long long n, int cout, const Norm nm,
                           float* loss) {
  __shared__ float red[256];
  float s = 0.f;
  const float inv = 1.0f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = (y[i] - t[i]) / nm.oscale[i % cout];
    s += d * d;
    if (dy) dy[i] = 2.0f * d * inv;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// Adam (bias-corrected) on the FP32 master weights
__global__ void adam_kernel(float* w, const float* gr, float* m, float* v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// WT (FP32 master, [co][tap*cin + ci]) -> BF16 WT and its transpose WD [ci][tap*cout + co]
// The BF16 copies of a convolution's weights w[co][tap][ci]: wt in the same
// order, wd transposed for the data gradient ([ci][tap][co]), and for the
// tcgen05 kernels wtp / wdp (either may be NULL) packed per K chunk of 16
// channels as [chunk][tap][half][n][8], n the output channel of the product
// (co for the forward, ci for the data gradient) and the 8 channels of the
// half contiguous: the weights of a chunk for a block of n are 18 runs of
// 16-byte rows, one box of one bulk tensor copy.
__global__ void weights_bf16_kernel(const float* w, __nv_bfloat16* wt, __nv_bfloat16* wd, __nv_bfloat16* wtp,
                                    __nv_bfloat16* wdp, int cout, int cin, int taps) {
  const long long n = (long long)cout * taps * cin;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(i / ((long long)taps * cin));
    const int k = (int)(i - (long long)co * taps * cin);
    const int tap = k / cin, ci = k - tap * cin;
    const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
    wt[i] = b;
    if (wd) wd[((size_t)ci * taps + tap) * cout + co] = b;
    if (wtp) wtp[(((size_t)(ci >> 4) * 18 + tap * 2 + ((ci >> 3) & 1)) * cout + co) * 8 + (ci & 7)] = b;
    if (wdp) wdp[(((size_t)(co >> 4) * 18 + tap * 2 + ((co >> 3) & 1)) * cin + ci) * 8 + (co & 7)] = b;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t conv_forward(const ConvArgs& a, cudaStream_t s) {
  if (a.tc && conv_tc_supported(a, 0)) return conv_forward_tc(a, s);
  dim3 grid((a.npix + BM - 1) / BM, (a.cout + 63) / 64);
  if (a.cout % 64 == 0) {
    igemm_kernel<0, 64><<<grid, NT, 0, s>>>(a);
  } else {
    grid.y = (a.cout + 31) / 32;
    igemm_kernel<0, 32><<<grid, NT, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t conv_dgrad(const ConvArgs& a, cudaStream_t s) {
  if (a.tc && conv_tc_supported(a, 1)) return conv_dgrad_tc(a, s);
  dim3 grid((a.npix + BM - 1) / BM, (a.cin + 63) / 64);
  if (a.cin % 64 == 0) {
    igemm_kernel<1, 64><<<grid, NT, 0, s>>>(a);
  } else {
    grid.y = (a.cin + 31) / 32;
    igemm_kernel<1, 32><<<grid, NT, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t conv_wgrad(const ConvArgs& a, cudaStream_t s) {
  const int ks = a.taps == 9 ? 9 : 1;
  dim3 grid((a.cout + BM - 1) / BM, (ks * a.cin + 63) / 64, (a.npix + a.ksplit - 1) / a.ksplit);
  igemm_kernel<2, 64><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t dsilu_bias(const __nv_bfloat16* dy, int ldy, int yoff, const __nv_bfloat16* z, __nv_bfloat16* dz,
                       long long npix, int c, float* db, cudaStream_t s) {
  const int G = c / 8;
  const int lanes = G >= 256 ? 1 : 256 / G;
  long long nb = (npix + lanes - 1) / lanes;
  if (nb > 152 * 8) nb = 152 * 8;
  dsilu_bias_kernel<<<(unsigned)nb, G * lanes, c * sizeof(float), s>>>(dy, ldy, yoff, z, dz, npix, c, db);
  return cudaGetLastError();
}

cudaError_t pool_fwd(const __nv_bfloat16* x, int ldx, int xoff, __nv_bfloat16* y, int B, int H, int W, int c,
                     cudaStream_t s) {
  pool_fwd_kernel<<<blocks_for((long long)B * H * W * c / 32), 256, 0, s>>>(x, ldx, xoff, y, B, H, W, c);
  return cudaGetLastError();
}

cudaError_t pool_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int ldx, int xoff, int B, int H, int W, int c,
                     int accumulate, cudaStream_t s) {
  pool_bwd_kernel<<<blocks_for((long long)B * H * W * c / 8), 256, 0, s>>>(dy, dx, ldx, xoff, B, H, W, c, accumulate);
  return cudaGetLastError();
}

cudaError_t up_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int B, int H, int W, int c, cudaStream_t s) {
  up_bwd_kernel<<<blocks_for((long long)B * H * W * c / 32), 256, 0, s>>>(dy, dx, B, H, W, c);
  return cudaGetLastError();
}

cudaError_t copy_ch(const __nv_bfloat16* src, int lds, int soff, __nv_bfloat16* dst, int ldd, int doff, long long npix,
                    int c, int accumulate, cudaStream_t s) {
  copy_ch_kernel<<<blocks_for(npix * c / 8), 256, 0, s>>>(src, lds, soff, dst, ldd, doff, npix, c, accumulate);
  return cudaGetLastError();
}

cudaError_t to_bf16(const float* x, int cin, __nv_bfloat16* y, int ldo, long long npix, const Norm& nm,
                    cudaStream_t s) {
  if (ldo == 16 && cin <= 16 && (reinterpret_cast<uintptr_t>(y) & 15) == 0)
    to_bf16_16_kernel<<<blocks_for(npix), 256, 0, s>>>(x, cin, y, npix, nm);
  else
    to_bf16_kernel<<<blocks_for(npix * ldo), 256, 0, s>>>(x, cin, y, ldo, npix, nm);
  return cudaGetLastError();
}

cudaError_t head_fwd(const __nv_bfloat16* x, int cin, const float* w, const float* b, float* y, int cout,
                     long long npix, const float* xin, int in_ch, const Norm& nm, cudaStream_t s) {
  head_fwd_kernel<<<blocks_for(npix), 256, (cout * cin + cout) * sizeof(float), s>>>(x, cin, w, b, y, cout, npix,
                                                                                      xin, in_ch, nm);
  return cudaGetLastError();
}

cudaError_t head_bwd(const __nv_bfloat16* x, int cin, const float* w, const float* dy, int cout, __nv_bfloat16* dx,
                     float* dw, float* db, long long npix, cudaStream_t s) {
  int TP = 8192 / cin;
  if (TP > 256) TP = 256;
  if (TP < 8) TP = 8;
  const size_t nf = (size_t)((cout * cin + cout + cout * cin + TP * cout + 3) & ~3);
  const size_t smem = nf * sizeof(float) + (size_t)TP * cin * 2;
  long long nb = (npix + TP - 1) / TP;
  if (nb > 152 * 4) nb = 152 * 4;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(head_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  head_bwd_kernel<<<(unsigned)nb, 256, smem, s>>>(x, cin, w, dy, cout, dx, dw, db, npix, TP);
  return cudaGetLastError();
}

cudaError_t mse(const float* y, const float* t, float* dy, long long n, int cout, const Norm& nm, float* loss,
                cudaStream_t s) {
  mse_kernel<<<blocks_for(n), 256, 0, s>>>(y, t, dy, n, cout, nm, loss);
  return cudaGetLastError();
}

cudaError_t adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t s) {
  adam_kernel<<<blocks_for(n), 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t weights_bf16(const float* w, __nv_bfloat16* wt, __nv_bfloat16* wd, __nv_bfloat16* wtp,
                         __nv_bfloat16* wdp, int cout, int cin, int taps, cudaStream_t s) {
  const bool packable = taps == 9 && cin % 16 == 0 && cout % 16 == 0;
  weights_bf16_kernel<<<blocks_for((long long)cout * cin * taps), 256, 0, s>>>(
      w, wt, wd, packable ? wtp : nullptr, packable ? wdp : nullptr, cout, cin, taps);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace gpe2p
