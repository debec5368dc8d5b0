// conv_tc.cu -- the surrogate's 3x3 circular convolutions (forward and data
// gradient) as implicit GEMMs on the 5th-generation tensor cores.
//
// A work item is a tile of 128 output pixels (16 rows x 8 columns of one
// image: GEMM rows M = 128) for a block of BN output channels (GEMM columns
// N).  Its K dimension (tap, input channel) is walked in chunks of 16
// channels.  For a chunk the CTA stages:
//   A: the 18 x 10 input window of the tile (the 1-pixel halo wrapped
//      periodically), 16 channels, as no-swizzle K-major core matrices
//      [8-channel half][window row][window column][8 channels], by cp.async;
//   B: the weights of the 9 taps for those channels, [tap][half][n][8], by
//      bulk copies from weights packed per chunk in that order, unless the
//      CTA holds all its weights resident in shared memory.
// The A operand of tap (dy, dx) is the same window read from a start address
// shifted by (dy, dx) pixels: with 8-pixel tile rows, consecutive 8-row core
// matrices of M sit one window row (160 bytes) apart for every tap.  The 9
// tcgen05.mma of a chunk (kind::f16, BF16 in, FP32 accumulator in tensor
// memory) are issued by one thread and committed to the stage's mbarrier.
//
// The CTAs are persistent and warp-specialised: CTA (x, y) takes the
// output-channel block y and the tiles x, x + gridDim.x, ...; the chunks of
// its tiles stream through a ring of stages filled by two producer warps,
// consumed by the MMA thread, and the double-buffered accumulator is drained
// by four epilogue warps (tcgen05.ld, bias, SiLU, BF16 NHWC stores) while
// the tensor cores work on the next tile.  The producers form their source
// pointers once per tile, so that a chunk costs a thread a handful of copies.
//
// The forward input may be read as the nearest 2x upsampling of a tensor of
// half the resolution (a.up), which fuses the decoder's upsampling into the
// convolution that follows it.
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
constexpr int A_BYTES = 2 * WH * WW * 16;   // 5760
constexpr int HEAD = 1024;                  // barriers and the tensor-memory slot
constexpr int SMEM_MAX = 200 * 1024;

template <int BN>
struct Cfg {
  static constexpr int BCHUNK = 9 * 2 * BN * 16;   // weights of one chunk
  static constexpr int TCOLS = 2 * BN < 32 ? 32 : 2 * BN;   // two accumulators
};

__device__ __forceinline__ int wrapm(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// wait until every cp.async this thread has issued has completed
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// contiguous bulk copy global -> shared of `bytes` (a multiple of 16, both
// addresses 16-byte aligned), completion counted on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// a bounded wait that also gives up as soon as another role of the CTA has
// aborted (sleeping between polls when asked, for roles with nothing else to do)
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag, bool sleep) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag != 0 || clock64() - t0 > WAIT_CYCLES) return false;
    if (sleep) __nanosleep(128);
  }
  return true;
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

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128
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
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

struct TileGeom {
  int b, y0, x0;
};

__device__ __forceinline__ TileGeom tile_of(int t, int tiles_x, int tiles_y) {
  TileGeom g;
  const int tx = t % tiles_x;
  t /= tiles_x;
  g.y0 = (t % tiles_y) * TH;
  g.b = t / tiles_y;
  g.x0 = tx * TW;
  return g;
}

// ---------------------------------------------------------------------------
// the warp-specialised form: each warp has one role
// ---------------------------------------------------------------------------
//   warps 0-3: epilogue; warp w reads tensor-memory lanes 32w .. 32w + 31
//              (the pixels of its quarter of the tile), applies bias and SiLU
//              and stores BF16;
//   warps 4-5: producers; they stage the input window of each K chunk with
//              cp.async and (unless resident) its weights with bulk copies
//              into a ring of ns stages; each thread's copies arrive on the
//              stage's full barrier by themselves when they land
//              (cp.async.mbarrier.arrive.noinc), the bulk copies count their
//              bytes on it, so a producer waits only for a free stage and
//              keeps up to ns chunks in flight;
//   warp 6:    one thread waits for a full stage, fences it to the async
//              proxy, issues the chunk's tcgen05.mma and commits them to the
//              stage's empty barrier, and at a tile's last chunk to the
//              accumulator's full barrier.
// The accumulator is double-buffered in tensor memory; the epilogue frees a
// buffer (its empty barrier) as soon as it has read it.  Every wait is
// bounded: a wait that runs out sets an abort flag that every role polls, and
// the CTA records the error, lets its MMAs finish and frees its tensor memory.
constexpr int EPI_WARPS = 4, PROD_WARPS = 2;
constexpr int NTHR = 32 * (EPI_WARPS + PROD_WARPS + 1);
constexpr int MMA_WARP = EPI_WARPS + PROD_WARPS;
constexpr int SMIN = 2, SMAX = 8;  // stages of the ring (chosen per launch)
constexpr int MAX_OCC = 4;         // CTAs per SM at most

__host__ __device__ __forceinline__ int smem_bytes(int bn, int nchunks, bool resident, int ns) {
  const int bchunk = 9 * 2 * bn * 16;
  return 1024 + HEAD + ns * (A_BYTES + (resident ? 0 : bchunk)) + (resident ? nchunks * bchunk : 0);
}

// the mbarrier receives one arrival (counted in its expected count, "noinc")
// once every cp.async this thread has issued so far has completed
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// BF16 results of one tile from its accumulator at acc (columns acc .. acc + BN):
// forward y = act(z + bias) (and z), data gradient dx (+)= value; one pixel
// per epilogue thread (lane m of the tile)
template <int MODE, int BN>
__device__ __forceinline__ void epilogue_tile(const ConvArgs& a, uint32_t acc, const TileGeom& tg, int n0, int m,
                                            int warp) {
  const int y = tg.y0 + m / TW, x = tg.x0 + m % TW;
  const bool valid = y < a.H && x < a.W;
  const size_t p = ((size_t)tg.b * a.H + (valid ? y : 0)) * a.W + (valid ? x : 0);
#pragma unroll 1
  for (int j = 0; j < BN; j += 16) {
    uint32_t v[16];
    const uint32_t ta = acc + ((uint32_t)(warp * 32) << 16) + (uint32_t)j;
    tmem_ld8(ta, v);
    tmem_ld8(ta + 8, v + 8);
    tmem_wait_ld();
    if (!valid) continue;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int n = n0 + j + 8 * hh;
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) f[e] = __uint_as_float(v[8 * hh + e]);
      if (MODE == 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] += a.bias[n + e];  // the bias sits at any offset of the parameters
        if (a.z) {
          uint4 zz;
          __nv_bfloat162* zp = reinterpret_cast<__nv_bfloat162*>(&zz);
#pragma unroll
          for (int e = 0; e < 4; ++e) zp[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
          *reinterpret_cast<uint4*>(a.z + p * a.cout + n) = zz;
        }
        uint4 yv;
        __nv_bfloat162* yp = reinterpret_cast<__nv_bfloat162*>(&yv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float u0 = a.act ? silu_f(f[2 * e]) : f[2 * e];
          const float u1 = a.act ? silu_f(f[2 * e + 1]) : f[2 * e + 1];
          yp[e] = __floats2bfloat162_rn(u0, u1);
        }
        *reinterpret_cast<uint4*>(a.y + p * a.ldy + a.yoff + n) = yv;
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
}

template <int MODE, int BN>
__global__ void __launch_bounds__(NTHR) conv3_tc_kernel(const ConvArgs a, int tiles_x, int tiles_y, int ntiles,
                                                       int resident, int ns) {
  using C = Cfg<BN>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);   // ns: a stage's copies landed (the producers arrive)
  uint64_t* empty = full + SMAX;                   // ns: a stage's MMAs finished (tcgen05.commit)
  uint64_t* accf = empty + SMAX;                     // 2: an accumulator's tile is complete (tcgen05.commit)
  uint64_t* acce = accf + 2;                          // 2: an accumulator has been read (the epilogue arrives)
  uint64_t* wbar = acce + 2;                          // the resident weights have landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 512);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + 520);
  unsigned char* stages = sm + HEAD;
  const int stage_bytes = A_BYTES + (resident ? 0 : C::BCHUNK);
  unsigned char* wres = stages + ns * stage_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int n0 = blockIdx.y * BN;
  const int H = a.H, W = a.W;
  const int Hs = a.up ? H >> 1 : H, Ws = a.up ? W >> 1 : W;
  const int Cin = MODE == 0 ? a.cin : a.cout;
  const __nv_bfloat16* src = MODE == 0 ? a.x : a.dz;
  const int lds = MODE == 0 ? a.ldx : a.ldz;
  const int soff = MODE == 0 ? a.xoff : 0;
  const int nchunks = Cin / KC;
  const int nout_all = MODE == 0 ? a.cout : a.cin;  // rows of the packed weights
  const int nitems = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int G = nitems * nchunks;

  // the next kernel on the stream may start its own set-up now; it reads
  // this kernel's outputs only after its grid-dependency wait
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 32 * PROD_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 32 * EPI_WARPS);
    }
    mbar_init(wbar, 1);
    *abort_flag = 0;
    fence_mbar_init();
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

  if (warp >= EPI_WARPS && warp < MMA_WARP) {
    // ---- producers ----
    // thread pt copies the 8-channel half hq of the window entries r0 + 32 j,
    // from source pointers formed once per tile, so that a chunk costs it a
    // handful of copies.  The weights of a chunk come as 18 contiguous bulk
    // copies from the weights packed per chunk.
    const int pt = tid - 32 * EPI_WARPS;
    constexpr int NP = 32 * PROD_WARPS;
    static_assert(NP == 64, "two producer warps: 32 window entries per pass");
    constexpr int NWIN = (WH * WW + 31) / 32;
    const int hq = pt & 1, r0 = pt >> 1;
    // the weights of chunk kk into B ([tap][half][n][8]), counted on bar: the
    // packed weights hold each (tap, half) run of the block's BN output
    // channels as BN x 16 contiguous bytes, one bulk copy by lane q < 18 of
    // the first producer warp
    const __nv_bfloat16* wpk = MODE == 0 ? a.wtp : a.wdp;
    auto load_weights = [&](unsigned char* B, int kk, uint64_t* bar) {
      if (pt < 18)
        bulk_load(B + pt * BN * 16, wpk + (((size_t)kk * 18 + pt) * nout_all + n0) * 8, (uint32_t)(BN * 16), bar);
    };
    const __nv_bfloat16* wp[NWIN];  // this tile's window sources of this thread (channel 0 of its half)
    if (resident && G > 0 && pt < 32) {
      if (pt == 0) mbar_arrive_expect_tx(wbar, (uint32_t)(nchunks * C::BCHUNK));
      __syncwarp();  // the bytes are announced before any of them can land
      for (int kk = 0; kk < nchunks; ++kk) load_weights(wres + kk * C::BCHUNK, kk, wbar);
    }
    // the window is the previous kernel's output: wait until that kernel has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int s = 0, k = 0, item = 0;
    uint32_t epar = 1;  // parity of the empty phase a stage's next use waits for (none in the first round)
    for (int g = 0; g < G; ++g) {
      // the warp leaves together (its lanes meet at __syncwarp below)
      bool stop = *abort_flag != 0;
      if (!stop && g >= ns) stop = !wait_or_abort(&empty[s], epar, abort_flag, true);
      if (__any_sync(0xffffffffu, stop)) {
        *abort_flag = 1;
        break;
      }
      if (k == 0) {
        const TileGeom tg = tile_of(blockIdx.x + item * gridDim.x, tiles_x, tiles_y);
#pragma unroll
        for (int j = 0; j < NWIN; ++j) {
          const int r = r0 + 32 * j;
          const int wy = r / WW, wx = r - wy * WW;
          int yy = wrapm(tg.y0 + wy - 1, H), xx = wrapm(tg.x0 + wx - 1, W);
          if (a.up) { yy >>= 1; xx >>= 1; }
          wp[j] = src + ((size_t)(tg.b * Hs + yy) * Ws + xx) * lds + soff + 8 * hq;
        }
      }
      unsigned char* A = stages + s * stage_bytes;
      const int c0 = k * KC;
      if (!resident && pt < 32) {
        // the bytes are announced before any of them can land, and before this
        // thread's own arrival below can complete the phase
        if (pt == 0) mbar_expect_tx(&full[s], (uint32_t)C::BCHUNK);
        __syncwarp();
        load_weights(A + A_BYTES, k, &full[s]);
      }
      unsigned char* da = A + (hq * WH * WW + r0) * 16;
#pragma unroll
      for (int j = 0; j < NWIN; ++j)
        if (r0 + 32 * j < WH * WW) cp_async16(da + 512 * j, wp[j] + c0);
      // the stage's full barrier receives this thread's arrival once every
      // window copy it has issued so far has landed
      cp_async_arrive_noinc(&full[s]);
      if (++s == ns) { s = 0; epar ^= 1u; }
      if (++k == nchunks) { k = 0; ++item; }
    }
    cp_async_wait_all();  // no copy may be in flight when the CTA exits
  } else if (warp == MMA_WARP) {
    // ---- the MMA issuer ----
    // no stage can fill before the previous kernel completes: wait for it
    // here rather than by polling the first stage's barrier meanwhile
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (lane == 0 && G > 0) {
      // stage s, its use parity fpar, chunk k of item: kept as counters (no divisions in the loop);
      // the descriptors are formed once per chunk, each tap adding a constant to the address field
      const uint32_t idesc = idesc_bf16<BN>();
      const uint64_t ad_lay = sdesc(0, WH * WW * 16, WW * 16), bd_lay = sdesc(0, BN * 16, 128);
      const uint32_t a_base = smem_u32(stages), w_base = smem_u32(wres);
      bool ok = !resident || wait_or_abort(wbar, 0, abort_flag, false);  // the resident weights
      int s = 0, k = 0, item = 0;
      uint32_t fpar = 0;
      for (int g = 0; g < G && ok; ++g) {
        if (*abort_flag) { ok = false; break; }
        const int buf = item & 1;
        // the buffer's tile of two items ago has been read by the epilogue
        if (k == 0 && item >= 2 && !wait_or_abort(&acce[buf], (uint32_t)(((item - 2) >> 1) & 1), abort_flag, false)) {
          ok = false;
          break;
        }
        if (!wait_or_abort(&full[s], fpar, abort_flag, false)) { ok = false; break; }
        // test switch: the first filled stage is reported as lost (its copies have all landed)
        if (g == 0 && a.wait_fault) { ok = false; break; }
        // the window was written through the generic proxy (cp.async); the MMAs read it through the async proxy
        fence_proxy_async_smem();
        tc_fence_after();
        const uint32_t Aa = a_base + (uint32_t)(s * stage_bytes);
        const uint32_t Ba = resident ? w_base + (uint32_t)(k * C::BCHUNK) : Aa + A_BYTES;
        const uint64_t ad0 = ad_lay | ((Aa & 0x3FFFFu) >> 4), bd0 = bd_lay | ((Ba & 0x3FFFFu) >> 4);
        const uint32_t acc = tmem + (uint32_t)(buf * BN);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          int dy = tap / 3 - 1, dx = tap % 3 - 1;
          if (MODE == 1) { dy = -dy; dx = -dx; }
          const uint32_t aoff = (uint32_t)(((dy + 1) * WW + (dx + 1)) * 16) >> 4;
          const uint32_t boff = (uint32_t)(tap * 2 * BN * 16) >> 4;
          mma_tc(acc, ad0 + aoff, bd0 + boff, idesc, (k > 0 || tap > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
        if (k == nchunks - 1) mma_commit(&accf[buf]);
        if (++s == ns) { s = 0; fpar ^= 1u; }
        if (++k == nchunks) { k = 0; ++item; }
      }
      if (!ok) *abort_flag = 1;
    }
  } else {
    // ---- epilogue: warp w holds tensor-memory lanes 32w .. 32w + 31 ----
    // its stores (and the data gradient's reads of dx) follow the previous kernel
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int item = 0; item < nitems; ++item) {
      const int buf = item & 1;
      const bool ok = wait_or_abort(&accf[buf], (uint32_t)((item >> 1) & 1), abort_flag, true);
      // every lane of the warp takes the same branch before the aligned tensor-memory loads
      if (!__all_sync(0xffffffffu, ok ? 1 : 0) || __any_sync(0xffffffffu, *abort_flag != 0)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const TileGeom tg = tile_of(blockIdx.x + item * gridDim.x, tiles_x, tiles_y);
      epilogue_tile<MODE, BN>(a, tmem + (uint32_t)(buf * BN), tg, n0, warp * 32 + lane, warp);
      tc_fence_before();
      mbar_arrive(&acce[buf]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0 && a.err) atomicExch(a.err, 1);
    // give the MMAs and the weight copies issued so far a bounded time to
    // finish before the tensor memory and the shared memory are released
    const long long t0 = clock64();
    while (clock64() - t0 < 1000000) {}
  }
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS) : "memory");
  }
}

template <int MODE, int BN>
cudaError_t launch_tc(const ConvArgs& a, int tiles_x, int tiles_y, int ntiles, int nout, cudaStream_t s) {
  static int attr_set = 0;
  auto k = conv3_tc_kernel<MODE, BN>;
  cudaError_t e;
  if (!attr_set) {
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_MAX)) != cudaSuccess) return e;
    attr_set = 1;
  }
  const int nch = (MODE == 0 ? a.cin : a.cout) / KC;
  int dev = 0, nsm = 152, sm_smem = 233472, reserved = 1024;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  // Up to MAX_OCC CTAs per SM as the tensor memory and shared memory allow,
  // each with a ring of at least SMIN stages: a CTA issues its MMAs from one
  // thread, at most one per 53 cycles (gpe2p_mma_rate), while the SM takes
  // one every 40 (N = 32), 48 (N = 64) or 64 (N = 128) cycles from several
  // issuers, so the tensor pipe is kept busy only by several issuing CTAs.
  // The weights stay resident
  // if that still leaves the ring, else they stream through it; the ring
  // takes as many stages as fit (up to SMAX).
  const int tm_occ = 512 / Cfg<BN>::TCOLS;
  bool resident = false;
  int ns = 0, occ = 1;
  for (int want = tm_occ < MAX_OCC ? tm_occ : MAX_OCC; want >= 1 && ns == 0; --want) {
    int budget = sm_smem / want - reserved;
    if (budget > SMEM_MAX) budget = SMEM_MAX;
    if (smem_bytes(BN, nch, true, SMIN) <= budget) {
      resident = true;
      ns = SMIN;
      while (ns < SMAX && smem_bytes(BN, nch, true, ns + 1) <= budget) ++ns;
    } else if (smem_bytes(BN, nch, false, SMIN) <= budget) {
      ns = SMIN;
      while (ns < SMAX && smem_bytes(BN, nch, false, ns + 1) <= budget) ++ns;
    }
    occ = want;
  }
  if (ns == 0) return cudaErrorInvalidValue;
  const int smem = smem_bytes(BN, nch, resident, ns);
  const int nblk_n = nout / BN;
  long long gx = ((long long)occ * nsm + nblk_n - 1) / nblk_n;
  if (gx > ntiles) gx = ntiles;
  if (gx < 1) gx = 1;
  dim3 grid((unsigned)gx, (unsigned)nblk_n);
  // Programmatic dependent launch where a CTA has at most two work items
  // (small batches, the deep levels): its set-up (barriers, tensor memory,
  // resident weights) then overlaps the tail of the kernel before it.  With
  // many items per CTA there is little tail to overlap, and the early
  // launch measured slower.  The kernel's grid-dependency instructions are
  // no-ops when it is launched without the attribute.
  const bool pdl = (ntiles + gx - 1) / gx <= 2;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a, tiles_x, tiles_y, ntiles, resident ? 1 : 0, ns);
}

template <int MODE>
cudaError_t conv3_tc(const ConvArgs& a, cudaStream_t s) {
  const int nout = MODE == 0 ? a.cout : a.cin;
  const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
  const long long tiles = (long long)a.B * tiles_x * tiles_y;
  if (tiles > (1LL << 30)) return cudaErrorInvalidValue;
  // the widest block of output channels (up to 128) that still gives every
  // SM a work item: a wider N does the same work in fewer MMAs (one thread
  // issues at most one per 53 cycles whatever N) and reads each window for
  // more outputs
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int bn = 128;
  while (bn > 16 && nout % bn) bn >>= 1;
  while (bn > 32 && tiles * (nout / bn) < nsm) bn >>= 1;
  switch (bn) {
    case 128: return launch_tc<MODE, 128>(a, tiles_x, tiles_y, (int)tiles, nout, s);
    case 64: return launch_tc<MODE, 64>(a, tiles_x, tiles_y, (int)tiles, nout, s);
    case 32: return launch_tc<MODE, 32>(a, tiles_x, tiles_y, (int)tiles, nout, s);
    default: return launch_tc<MODE, 16>(a, tiles_x, tiles_y, (int)tiles, nout, s);
  }
}

}  // namespace

bool conv_tc_supported(const ConvArgs& a, int mode) {
  const int kin = mode == 0 ? a.cin : a.cout, nout = mode == 0 ? a.cout : a.cin;
  if (a.taps != 9 || kin % KC || nout % 16 || a.H < 1 || a.W < 1) return false;
  if (mode == 0 && a.up && (a.H % 2 || a.W % 2)) return false;
  if (mode == 1 && a.up) return false;
  const int ld = mode == 0 ? a.ldx : a.ldz, off = mode == 0 ? a.xoff : 0;
  const int ldo = mode == 0 ? a.ldy : a.lddx, offo = mode == 0 ? a.yoff : a.dxoff;
  if (smem_bytes(16, kin / KC, false, SMIN) > SMEM_MAX) return false;
  if (!(mode == 0 ? a.wtp : a.wdp)) return false;  // the weights packed per K chunk
  return ld % 8 == 0 && off % 8 == 0 && ldo % 8 == 0 && offo % 8 == 0;
}

cudaError_t conv_forward_tc(const ConvArgs& a, cudaStream_t s) { return conv3_tc<0>(a, s); }
cudaError_t conv_dgrad_tc(const ConvArgs& a, cudaStream_t s) { return conv3_tc<1>(a, s); }

}  // namespace nn
}  // namespace gpe2p
