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
          const int yy = wrapi(y + dy, a.H), xx = wrapi(x + dx, a.W);
          const __nv_bfloat16* src = MODE == 0 ? a.x : a.dz;
          const int ld = MODE == 0 ? a.ldx : a.ldz;
          const int off = MODE == 0 ? a.xoff : 0;
          const uint4* s = reinterpret_cast<const uint4*>(src + ((size_t)(b * a.H + yy) * a.W + xx) * ld + off + c);
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
          const int yy = wrapi(y + dy, a.H), xx = wrapi(x + dx, a.W);
          v = *reinterpret_cast<const uint4*>(a.x + ((size_t)(b * a.H + yy) * a.W + xx) * a.ldx + a.xoff + ci);
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

// dZ = dY * silu'(z) (dY read with row stride ldy and channel offset yoff)
__global__ void dsilu_kernel(const __nv_bfloat16* dy, int ldy, int yoff, const __nv_bfloat16* z, __nv_bfloat16* dz,
                             long long npix, int c) {
  const long long n = npix * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / c;
    const int ch = (int)(i - p * c);
    const float g = __bfloat162float(dy[p * ldy + yoff + ch]);
    dz[i] = __float2bfloat16_rn(g * dsilu(__bfloat162float(z[i])));
  }
}

// db[c] += sum_p dZ[p, c]
__global__ void bias_grad_kernel(const __nv_bfloat16* dz, long long npix, int c, float* db) {
  extern __shared__ float red[];
  for (int ch = threadIdx.x; ch < c; ch += blockDim.x) red[ch] = 0.f;
  __syncthreads();
  for (long long p = blockIdx.x; p < npix; p += gridDim.x)
    for (int ch = threadIdx.x; ch < c; ch += blockDim.x) red[ch] += __bfloat162float(dz[p * c + ch]);
  __syncthreads();
  for (int ch = threadIdx.x; ch < c; ch += blockDim.x) atomicAdd(db + ch, red[ch]);
}

// 2x2 average pooling (forward) and its adjoint
__global__ void pool_fwd_kernel(const __nv_bfloat16* x, int ldx, int xoff, __nv_bfloat16* y, int B, int H, int W,
                                int c) {
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)B * Ho * Wo * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long q = i / c;
    const int xo = (int)(q % Wo);
    q /= Wo;
    const int yo = (int)(q % Ho);
    const int b = (int)(q / Ho);
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        s += __bfloat162float(x[((size_t)(b * H + 2 * yo + dy) * W + 2 * xo + dx) * ldx + xoff + ch]);
    y[i] = __float2bfloat16_rn(0.25f * s);
  }
}

// dX (row stride ldx, offset xoff) = 1/4 dY spread; accumulate adds to dX
__global__ void pool_bwd_kernel(const __nv_bfloat16* dy, __nv_bfloat16* dx, int ldx, int xoff, int B, int H, int W,
                                int c, int accumulate) {
  const long long n = (long long)B * H * W * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long q = i / c;
    const int x = (int)(q % W);
    q /= W;
    const int y = (int)(q % H);
    const int b = (int)(q / H);
    const float g = 0.25f * __bfloat162float(dy[((size_t)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * c + ch]);
    __nv_bfloat16* d = dx + ((size_t)(b * H + y) * W + x) * ldx + xoff + ch;
    *d = __float2bfloat16_rn(accumulate ? g + __bfloat162float(*d) : g);
  }
}

// nearest-neighbour 2x upsampling and its adjoint (sum of the four children)
__global__ void up_fwd_kernel(const __nv_bfloat16* x, __nv_bfloat16* y, int B, int H, int W, int c) {
  const long long n = (long long)B * H * W * c;  // H, W of the output
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long q = i / c;
    const int xx = (int)(q % W);
    q /= W;
    const int yy = (int)(q % H);
    const int b = (int)(q / H);
    y[i] = x[((size_t)(b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * c + ch];
  }
}

__global__ void up_bwd_kernel(const __nv_bfloat16* dy, __nv_bfloat16* dx, int B, int H, int W, int c) {
  const int Hi = H / 2, Wi = W / 2;  // H, W of dY
  const long long n = (long long)B * Hi * Wi * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long q = i / c;
    const int xo = (int)(q % Wi);
    q /= Wi;
    const int yo = (int)(q % Hi);
    const int b = (int)(q / Hi);
    float s = 0.f;
    for (int dy2 = 0; dy2 < 2; ++dy2)
      for (int dx2 = 0; dx2 < 2; ++dx2) s += __bfloat162float(dy[((size_t)(b * H + 2 * yo + dy2) * W + 2 * xo + dx2) * c + ch]);
    dx[i] = __float2bfloat16_rn(s);
  }
}

// copy c channels from (src, lds, soff) to (dst, ldd, doff); accumulate adds
__global__ void copy_ch_kernel(const __nv_bfloat16* src, int lds, int soff, __nv_bfloat16* dst, int ldd, int doff,
                               long long npix, int c, int accumulate) {
  const long long n = npix * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / c;
    const int ch = (int)(i - p * c);
    const float v = __bfloat162float(src[p * lds + soff + ch]);
    __nv_bfloat16* d = dst + p * ldd + doff + ch;
    *d = __float2bfloat16_rn(accumulate ? v + __bfloat162float(*d) : v);
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

// output layer: 1x1 convolution cin -> cout (small cout), FP32 out, no activation, then the
// output map (scale, optional residual from the raw FP32 input xin of in_ch channels)
__global__ void head_fwd_kernel(const __nv_bfloat16* x, int cin, const float* w, const float* b, float* y, int cout,
                                long long npix, const float* xin, int in_ch, const Norm nm) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    for (int o = 0; o < cout; ++o) {
      float s = b[o];
      for (int c = 0; c < cin; ++c) s += w[o * cin + c] * __bfloat162float(x[p * cin + c]);
      y[p * cout + o] = (nm.residual ? xin[p * in_ch + o] : 0.f) + nm.oscale[o] * s;
    }
  }
}

// its adjoint: dX = dY W (bf16), dW += sum_p dY x^T, db += sum_p dY
__global__ void head_bwd_kernel(const __nv_bfloat16* x, int cin, const float* w, const float* dy, int cout,
                                __nv_bfloat16* dx, float* dw, float* db, long long npix) {
  extern __shared__ float sred[];  // cout*cin + cout
  const int nr = cout * cin + cout;
  for (int q = threadIdx.x; q < nr; q += blockDim.x) sred[q] = 0.f;
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < cin; ++c) {
      float s = 0.f;
      for (int o = 0; o < cout; ++o) s += dy[p * cout + o] * w[o * cin + c];
      dx[p * cin + c] = __float2bfloat16_rn(s);
    }
    for (int o = 0; o < cout; ++o) {
      const float g = dy[p * cout + o];
      atomicAdd(&sred[cout * cin + o], g);
      for (int c = 0; c < cin; ++c) atomicAdd(&sred[o * cin + c], g * __bfloat162float(x[p * cin + c]));
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < cout * cin; q += blockDim.x) atomicAdd(dw + q, sred[q]);
  for (int q = threadIdx.x; q < cout; q += blockDim.x) atomicAdd(db + q, sred[cout * cin + q]);
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
__global__ void weights_bf16_kernel(const float* w, __nv_bfloat16* wt, __nv_bfloat16* wd, int cout, int cin, int taps) {
  const long long n = (long long)cout * taps * cin;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(i / ((long long)taps * cin));
    const int k = (int)(i - (long long)co * taps * cin);
    const int tap = k / cin, ci = k - tap * cin;
    const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
    wt[i] = b;
    if (wd) wd[((size_t)ci * taps + tap) * cout + co] = b;
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

cudaError_t dsilu(const __nv_bfloat16* dy, int ldy, int yoff, const __nv_bfloat16* z, __nv_bfloat16* dz,
                  long long npix, int c, cudaStream_t s) {
  dsilu_kernel<<<blocks_for(npix * c), 256, 0, s>>>(dy, ldy, yoff, z, dz, npix, c);
  return cudaGetLastError();
}

cudaError_t bias_grad(const __nv_bfloat16* dz, long long npix, int c, float* db, cudaStream_t s) {
  long long nb = npix / 256;
  if (nb < 1) nb = 1;
  if (nb > 152 * 4) nb = 152 * 4;
  bias_grad_kernel<<<(unsigned)nb, 128, c * sizeof(float), s>>>(dz, npix, c, db);
  return cudaGetLastError();
}

cudaError_t pool_fwd(const __nv_bfloat16* x, int ldx, int xoff, __nv_bfloat16* y, int B, int H, int W, int c,
                     cudaStream_t s) {
  pool_fwd_kernel<<<blocks_for((long long)B * H * W * c / 4), 256, 0, s>>>(x, ldx, xoff, y, B, H, W, c);
  return cudaGetLastError();
}

cudaError_t pool_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int ldx, int xoff, int B, int H, int W, int c,
                     int accumulate, cudaStream_t s) {
  pool_bwd_kernel<<<blocks_for((long long)B * H * W * c), 256, 0, s>>>(dy, dx, ldx, xoff, B, H, W, c, accumulate);
  return cudaGetLastError();
}

cudaError_t up_fwd(const __nv_bfloat16* x, __nv_bfloat16* y, int B, int H, int W, int c, cudaStream_t s) {
  up_fwd_kernel<<<blocks_for((long long)B * H * W * c), 256, 0, s>>>(x, y, B, H, W, c);
  return cudaGetLastError();
}

cudaError_t up_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int B, int H, int W, int c, cudaStream_t s) {
  up_bwd_kernel<<<blocks_for((long long)B * H * W * c / 4), 256, 0, s>>>(dy, dx, B, H, W, c);
  return cudaGetLastError();
}

cudaError_t copy_ch(const __nv_bfloat16* src, int lds, int soff, __nv_bfloat16* dst, int ldd, int doff, long long npix,
                    int c, int accumulate, cudaStream_t s) {
  copy_ch_kernel<<<blocks_for(npix * c), 256, 0, s>>>(src, lds, soff, dst, ldd, doff, npix, c, accumulate);
  return cudaGetLastError();
}

cudaError_t to_bf16(const float* x, int cin, __nv_bfloat16* y, int ldo, long long npix, const Norm& nm,
                    cudaStream_t s) {
  to_bf16_kernel<<<blocks_for(npix * ldo), 256, 0, s>>>(x, cin, y, ldo, npix, nm);
  return cudaGetLastError();
}

cudaError_t head_fwd(const __nv_bfloat16* x, int cin, const float* w, const float* b, float* y, int cout,
                     long long npix, const float* xin, int in_ch, const Norm& nm, cudaStream_t s) {
  head_fwd_kernel<<<blocks_for(npix), 256, 0, s>>>(x, cin, w, b, y, cout, npix, xin, in_ch, nm);
  return cudaGetLastError();
}

cudaError_t head_bwd(const __nv_bfloat16* x, int cin, const float* w, const float* dy, int cout, __nv_bfloat16* dx,
                     float* dw, float* db, long long npix, cudaStream_t s) {
  long long nb = (npix + 255) / 256;
  if (nb > 152 * 4) nb = 152 * 4;
  head_bwd_kernel<<<(unsigned)nb, 256, (cout * cin + cout) * sizeof(float), s>>>(x, cin, w, dy, cout, dx, dw, db,
                                                                                  npix);
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

cudaError_t weights_bf16(const float* w, __nv_bfloat16* wt, __nv_bfloat16* wd, int cout, int cin, int taps,
                         cudaStream_t s) {
  weights_bf16_kernel<<<blocks_for((long long)cout * cin * taps), 256, 0, s>>>(w, wt, wd, cout, cin, taps);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace gpe2p
