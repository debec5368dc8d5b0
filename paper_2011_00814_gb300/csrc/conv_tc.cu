// conv_tc.cu -- the surrogate's 3x3 circular convolutions (forward and data
// gradient) as implicit GEMMs on the 5th-generation tensor cores.
//
// One CTA computes a tile of 128 output pixels (16 rows x 8 columns of one
// image: GEMM rows M = 128) for BN output channels (GEMM columns N).  The K
// dimension (tap, input channel) is walked in chunks of 16 channels.  For a
// chunk the CTA stages, with cp.async:
//   A: the 18 x 10 input window of the tile (the 1-pixel halo wrapped
//      periodically), 16 channels, as no-swizzle K-major core matrices
//      [8-channel half][window row][window column][8 channels];
//   B: the weights of the 9 taps for those channels, [tap][half][n][8].
// The A operand of tap (dy, dx) is the same window read from a start address
// shifted by (dy, dx) pixels: with 8-pixel tile rows, consecutive 8-row core
// matrices of M sit one window row (160 bytes) apart for every tap.  One
// thread issues the 9 tcgen05.mma (kind::f16, BF16 in, FP32 accumulator in
// tensor memory) of a chunk and commits them to the chunk's mbarrier; the
// stage is refilled only after that barrier completes.  The epilogue reads
// the accumulator with tcgen05.ld (one pixel row per thread), adds the bias,
// applies SiLU and stores BF16 NHWC.
//
// Every wait is bounded (about 2 s of SM clock); on a timeout the CTA records
// an error in a.err, stops issuing work, waits (bounded) for its MMAs and
// frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn.h"
#include "tma.cuh"

namespace gpe2p {
namespace nn {
namespace {

constexpr int TH = 16, TW = 8;              // output tile (M = 128 pixels)
constexpr int WH = TH + 2, WW = TW + 2;     // input window with the halo
constexpr int KC = 16;                      // channels per K chunk
constexpr int NTHR = 128;
constexpr int A_BYTES = 2 * WH * WW * 16;   // 5760
// Room past the staged operands so that every address the descriptors can
// form stays inside the CTA's shared memory for either reading of the
// descriptor's two byte-offset fields.
constexpr int SLACK = 48 * 1024;

template <int BN>
struct Cfg {
  static constexpr int S = BN >= 128 ? 3 : 4;      // stages
  static constexpr int PD = S - 2;                 // chunks loaded ahead
  static constexpr int B_BYTES = 9 * 2 * BN * 16;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = 1024 + 1024 + S * STAGE + SLACK;   // alignment + barriers + stages + slack
  static constexpr int TCOLS = BN < 32 ? 32 : BN;  // tensor-memory columns (power of two >= 32)
};

__device__ __forceinline__ int wrapm(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups along M (or N)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
  return d;                // base offset 0, absolute lbo mode 0, layout 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
template <int N>
__device__ __forceinline__ uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tc(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t v[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }

// MODE 0: forward  y = act(conv(x) + bias) (and z = conv(x) + bias);
// MODE 1: data gradient  dx (+)= conv^T(dz)
template <int MODE, int BN>
__global__ void __launch_bounds__(NTHR, 1) conv3_tc_kernel(const ConvArgs a, int tiles_x, int tiles_y) {
  using C = Cfg<BN>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 512);
  unsigned char* stages = sm + 1024;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  int t = blockIdx.x;
  const int tx = t % tiles_x;
  t /= tiles_x;
  const int ty = t % tiles_y;
  const int b = t / tiles_y;
  const int y0 = ty * TH, x0 = tx * TW;
  const int n0 = blockIdx.y * BN;
  const int H = a.H, W = a.W;
  const int Cin = MODE == 0 ? a.cin : a.cout;     // channels of the K dimension
  const __nv_bfloat16* src = MODE == 0 ? a.x : a.dz;
  const int lds = MODE == 0 ? a.ldx : a.ldz;
  const int soff = MODE == 0 ? a.xoff : 0;
  const __nv_bfloat16* wsrc = MODE == 0 ? a.wt : a.wd;
  const int Kw = 9 * Cin;                          // row length of the weight matrix
  const int nchunks = Cin / KC;

  if (tid == 0) {
    for (int s = 0; s < C::S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  auto load_chunk = [&](int k, int s) {
    unsigned char* A = stages + s * C::STAGE;
    unsigned char* B = A + A_BYTES;
    const int c0 = k * KC;
    for (int q = tid; q < 2 * WH * WW; q += NTHR) {
      const int h = q & 1, r = q >> 1;
      const int wy = r / WW, wx = r - wy * WW;
      const int yy = wrapm(y0 + wy - 1, H), xx = wrapm(x0 + wx - 1, W);
      const __nv_bfloat16* g = src + ((size_t)(b * H + yy) * W + xx) * lds + soff + c0 + 8 * h;
      cp_async16(A + ((h * WH + wy) * WW + wx) * 16, g);
    }
    for (int q = tid; q < 9 * 2 * BN; q += NTHR) {
      const int h = q & 1, r = q >> 1;
      const int tap = r / BN, n = r - tap * BN;
      cp_async16(B + ((tap * 2 + h) * BN + n) * 16, wsrc + (size_t)(n0 + n) * Kw + tap * Cin + c0 + 8 * h);
    }
  };

  for (int k = 0; k < C::PD && k < nchunks; ++k) {
    load_chunk(k, k % C::S);
    cp_async_commit();
  }
  for (int k = nchunks; k < C::PD; ++k) cp_async_commit();

  bool bad = false;
  for (int k = 0; k < nchunks; ++k) {
    const int kn = k + C::PD;
    if (kn < nchunks) {
      const int sn = kn % C::S;
      bool to = false;
      if (kn >= C::S) to = !mbar_wait_bounded(&bar[sn], (uint32_t)(((kn - C::S) / C::S) & 1), WAIT_CYCLES);
      if (__syncthreads_or(to)) { bad = true; break; }
      load_chunk(kn, sn);
    }
    cp_async_commit();
    cp_async_wait<C::PD>();
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const int s = k % C::S;
      const uint32_t Aa = smem_u32(stages + s * C::STAGE);
      const uint32_t Ba = Aa + A_BYTES;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (MODE == 1) { dy = -dy; dx = -dx; }
        const uint64_t ad = sdesc(Aa + (uint32_t)(((dy + 1) * WW + (dx + 1)) * 16), WH * WW * 16, WW * 16);
        const uint64_t bd = sdesc(Ba + (uint32_t)(tap * 2 * BN * 16), BN * 16, 128);
        mma_tc(tmem, ad, bd, idesc_bf16<BN>(), (k > 0 || tap > 0) ? 1u : 0u);
      }
      mma_commit(&bar[s]);
    }
  }
  cp_async_wait<0>();

  // the last committed chunk covers every MMA issued before it
  bool done = false;
  if (nchunks > 0) {
    const int kl = bad ? -1 : nchunks - 1;
    if (kl >= 0) done = mbar_wait_bounded(&bar[kl % C::S], (uint32_t)((kl / C::S) & 1), WAIT_CYCLES);
  }
  if (__syncthreads_or(!done)) {
    if (tid == 0 && a.err) atomicExch(a.err, 1);
    // drain: give the MMAs issued so far a bounded time to finish before the memory is freed
    const long long t0 = clock64();
    while (clock64() - t0 < 1000000) {}
  } else {
    tc_fence_after();
    const int m = warp * 32 + lane;
    const int y = y0 + m / TW, x = x0 + m % TW;
    const bool valid = y < H && x < W;
    const size_t p = ((size_t)b * H + (valid ? y : 0)) * W + (valid ? x : 0);
#pragma unroll 1
    for (int j = 0; j < BN; j += 8) {
      uint32_t v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j, v);
      if (!valid) continue;
      const int n = n0 + j;
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) f[e] = __uint_as_float(v[e]);
      if (MODE == 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] += a.bias[n + e];
        if (a.z) {
          uint4 zz;
          __nv_bfloat162* zp = reinterpret_cast<__nv_bfloat162*>(&zz);
#pragma unroll
          for (int e = 0; e < 4; ++e) zp[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
          *reinterpret_cast<uint4*>(a.z + p * a.cout + n) = zz;
        }
        uint4 yy;
        __nv_bfloat162* yp = reinterpret_cast<__nv_bfloat162*>(&yy);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float u0 = a.act ? silu_f(f[2 * e]) : f[2 * e];
          const float u1 = a.act ? silu_f(f[2 * e + 1]) : f[2 * e + 1];
          yp[e] = __floats2bfloat162_rn(u0, u1);
        }
        *reinterpret_cast<uint4*>(a.y + p * a.ldy + a.yoff + n) = yy;
      } else {
        __nv_bfloat16* dst = a.dx + p * a.lddx + a.dxoff + n;
        if (a.accumulate) {
          const uint4 old = *reinterpret_cast<const uint4*>(dst);
          const __nv_bfloat162* op = reinterpret_cast<const __nv_bfloat162*>(&old);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 o = __bfloat1622float2(op[e]);
            f[2 * e] += o.x;
            f[2 * e + 1] += o.y;
          }
        }
        uint4 dd;
        __nv_bfloat162* dp = reinterpret_cast<__nv_bfloat162*>(&dd);
#pragma unroll
        for (int e = 0; e < 4; ++e) dp[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
        *reinterpret_cast<uint4*>(dst) = dd;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS) : "memory");
  }
}

template <int MODE, int BN>
cudaError_t launch_tc(const ConvArgs& a, int tiles_x, int tiles_y, long long tiles, int nout, cudaStream_t s) {
  static bool attr = false;
  auto k = conv3_tc_kernel<MODE, BN>;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<BN>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((unsigned)tiles, (unsigned)(nout / BN));
  k<<<grid, NTHR, Cfg<BN>::SMEM, s>>>(a, tiles_x, tiles_y);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t conv3_tc(const ConvArgs& a, cudaStream_t s) {
  const int nout = MODE == 0 ? a.cout : a.cin;
  const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
  const long long tiles = (long long)a.B * tiles_x * tiles_y;
  int bn = 128;
  while (bn > 16 && nout % bn) bn >>= 1;
  while (bn > 32 && tiles * (nout / bn) < 2 * 152) bn >>= 1;
  switch (bn) {
    case 128: return launch_tc<MODE, 128>(a, tiles_x, tiles_y, tiles, nout, s);
    case 64: return launch_tc<MODE, 64>(a, tiles_x, tiles_y, tiles, nout, s);
    case 32: return launch_tc<MODE, 32>(a, tiles_x, tiles_y, tiles, nout, s);
    default: return launch_tc<MODE, 16>(a, tiles_x, tiles_y, tiles, nout, s);
  }
}

}  // namespace

bool conv_tc_supported(const ConvArgs& a, int mode) {
  const int kin = mode == 0 ? a.cin : a.cout, nout = mode == 0 ? a.cout : a.cin;
  if (a.taps != 9 || kin % KC || nout % 16 || a.H < 1 || a.W < 1) return false;
  const int ld = mode == 0 ? a.ldx : a.ldz, off = mode == 0 ? a.xoff : 0;
  const int ldo = mode == 0 ? a.ldy : a.lddx, offo = mode == 0 ? a.yoff : a.dxoff;
  return ld % 8 == 0 && off % 8 == 0 && ldo % 8 == 0 && offo % 8 == 0;
}

cudaError_t conv_forward_tc(const ConvArgs& a, cudaStream_t s) { return conv3_tc<0>(a, s); }
cudaError_t conv_dgrad_tc(const ConvArgs& a, cudaStream_t s) { return conv3_tc<1>(a, s); }

}  // namespace nn
}  // namespace gpe2p
