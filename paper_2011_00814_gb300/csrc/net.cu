// net.cu -- the surrogate's network: a U-Net of L levels on the periodic 2D
// grid, with its forward and backward passes and Adam, run on the kernels of
// nn.cu; and its part of the C ABI (include/gpe2p.h, gpe2p_net_*).
//
// Architecture (levels l = 0 .. L-1, channels c_l, resolution H/2^l):
//   encoder  l: [pool 2x2 if l > 0] conv3x3 -> SiLU -> conv3x3 -> SiLU   (output e_l)
//   decoder  l = L-2 .. 0: upsample x2 -> conv3x3 (c_{l+1} -> c_l) -> SiLU,
//            concatenated with e_l, conv3x3 (2c_l -> c_l) -> SiLU -> conv3x3 -> SiLU
//   head     1x1 convolution c_0 -> out channels (no activation)
// The input (FP32, in channels) is padded with zero channels to 16.
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/gpe2p.h"
#include "nn.h"

using namespace gpe2p::nn;

namespace {

thread_local std::string g_net_error;

struct ConvL {
  int cin, cout, taps, level;
  long long w, b;                 // offsets of weights and bias in the flat parameters
  __nv_bfloat16* wt = nullptr;    // [cout][taps*cin]
  __nv_bfloat16* wd = nullptr;    // [cin][taps*cout]
  __nv_bfloat16* wtp = nullptr;   // wt and wd packed per K chunk for the tcgen05 kernels (3x3 only)
  __nv_bfloat16* wdp = nullptr;
  __nv_bfloat16* z = nullptr;     // pre-activation [npix][cout]
};

struct Act {                      // a BF16 activation and its gradient
  __nv_bfloat16* v = nullptr;
  __nv_bfloat16* g = nullptr;
  int c = 0, level = 0;
};

}  // namespace

struct gpe2p_net {
  int L = 0, in_ch = 0, out_ch = 0, H = 0, W = 0, maxB = 0;
  std::vector<int> ch;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<ConvL> conv;
  std::vector<int> enc_a, enc_b, up, dec_a, dec_b;   // indices into conv
  long long nparam = 0, head_w = 0, head_b = 0;
  float *P = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr;
  long long adam_t = 0;
  int use_tc = 1;                // 3x3 forward / data gradient on tcgen05
  int wait_fault = 0;            // test switch of the tcgen05 kernels (gpe2p_net_fault)
  // the inference forward captured in a CUDA graph for one (x, y, batch)
  cudaGraphExec_t fwd_exec = nullptr;
  const float* fwd_x = nullptr;
  float* fwd_y = nullptr;
  int fwd_b = 0;
  int* d_err = nullptr;          // device error word of the tcgen05 kernels
  int* h_err = nullptr;          // pinned copy
  Norm norm{};
  Act in16;
  std::vector<Act> ea, eb, pooled, upx, cat, da, db;
  __nv_bfloat16* dz = nullptr;   // scratch for one layer's dZ
  float* out = nullptr;          // FP32 network output [npix0][out_ch]
  float* dout = nullptr;
  float* loss = nullptr;         // device scalar
  float* loss_h = nullptr;       // pinned
  std::vector<void*> allocs;
  std::string err;
};

static void drop_forward_graph(gpe2p_net* n);

static int net_fail(gpe2p_net* n, int code, const std::string& m) {
  if (n) n->err = m;
  else g_net_error = m;
  return code;
}

#define NK(n, call, what)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return net_fail(n, GPE2P_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static long long npix_at(const gpe2p_net* n, int level, int B) {
  return (long long)B * (n->H >> level) * (n->W >> level);
}

template <typename T>
static cudaError_t nalloc(gpe2p_net* n, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
  if (e == cudaSuccess) n->allocs.push_back(*p);
  return e;
}

static int add_conv(gpe2p_net* n, int cin, int cout, int taps, int level) {
  ConvL c;
  c.cin = cin;
  c.cout = cout;
  c.taps = taps;
  c.level = level;
  c.w = n->nparam;
  n->nparam += (long long)cout * taps * cin;
  c.b = n->nparam;
  n->nparam += cout;
  n->conv.push_back(c);
  return (int)n->conv.size() - 1;
}

static cudaError_t refresh_bf16(gpe2p_net* n) {
  for (auto& c : n->conv) {
    cudaError_t e = weights_bf16(n->P + c.w, c.wt, c.wd, c.wtp, c.wdp, c.cout, c.cin, c.taps, n->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static ConvArgs conv_args(const gpe2p_net* n, const ConvL& c, int B) {
  ConvArgs a{};
  a.B = B;
  a.H = n->H >> c.level;
  a.W = n->W >> c.level;
  a.npix = (int)npix_at(n, c.level, B);
  a.cin = c.cin;
  a.cout = c.cout;
  a.taps = c.taps;
  a.wt = c.wt;
  a.wd = c.wd;
  a.wtp = c.wtp;
  a.wdp = c.wdp;
  a.bias = n->P + c.b;
  a.z = c.z;
  a.act = 1;
  a.ldz = c.cout;
  a.dw = n->G + c.w;
  a.ksplit = 2048;
  a.tc = n->use_tc;
  a.err = n->d_err;
  a.wait_fault = n->wait_fault;
  return a;
}

// forward of layer c from (x, ldx, xoff) into (y, ldy, yoff); the pre-activation is stored
// for training; up: x is stored at half resolution and read upsampled
static cudaError_t fwd(gpe2p_net* n, const ConvL& c, int B, const __nv_bfloat16* x, int ldx, int xoff,
                       __nv_bfloat16* y, int ldy, int yoff, bool train, int up = 0) {
  ConvArgs a = conv_args(n, c, B);
  a.x = x;
  a.ldx = ldx;
  a.xoff = xoff;
  a.up = up;
  a.y = y;
  a.ldy = ldy;
  a.yoff = yoff;
  if (!train) a.z = nullptr;
  return conv_forward(a, n->stream);
}

// backward of layer c: dY (gy, ldgy, gyoff) -> dZ -> dW, db and (if gx) dX into (gx, ldgx, gxoff);
// up: the layer's input x is stored at half resolution (gx is then at full resolution)
static cudaError_t bwd(gpe2p_net* n, const ConvL& c, int B, const __nv_bfloat16* x, int ldx, int xoff,
                       const __nv_bfloat16* gy, int ldgy, int gyoff, __nv_bfloat16* gx, int ldgx, int gxoff,
                       int accumulate, int up = 0) {
  const long long np = npix_at(n, c.level, B);
  cudaError_t e = dsilu_bias(gy, ldgy, gyoff, c.z, n->dz, np, c.cout, n->G + c.b, n->stream);
  if (e != cudaSuccess) return e;
  ConvArgs a = conv_args(n, c, B);
  a.x = x;
  a.ldx = ldx;
  a.xoff = xoff;
  a.up = up;
  a.dz = n->dz;
  if ((e = conv_wgrad(a, n->stream)) != cudaSuccess) return e;
  if (gx) {
    a.up = 0;
    a.dx = gx;
    a.lddx = ldgx;
    a.dxoff = gxoff;
    a.accumulate = accumulate;
    if ((e = conv_dgrad(a, n->stream)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The encoder output of level l < L-1 is written straight into the second
// half of the decoder's concatenation buffer cat[l] (channels c..2c), where
// the decoder reads it and the pooling of level l+1 takes it from; the
// decoder's upsampling is read inside the convolution that follows it.
static cudaError_t forward(gpe2p_net* n, const float* x, int B, bool train) {
  const int L = n->L;
  cudaError_t e = to_bf16(x, n->in_ch, n->in16.v, 16, npix_at(n, 0, B), n->norm, n->stream);
  if (e != cudaSuccess) return e;
  for (int l = 0; l < L; ++l) {
    const __nv_bfloat16* in = n->in16.v;
    int ldin = 16;
    if (l > 0) {
      const int cp = n->ch[l - 1];
      if ((e = pool_fwd(n->cat[l - 1].v, 2 * cp, cp, n->pooled[l - 1].v, B, n->H >> (l - 1), n->W >> (l - 1), cp,
                        n->stream)) != cudaSuccess)
        return e;
      in = n->pooled[l - 1].v;
      ldin = cp;
    }
    if ((e = fwd(n, n->conv[n->enc_a[l]], B, in, ldin, 0, n->ea[l].v, n->ch[l], 0, train)) != cudaSuccess) return e;
    const bool last = l == L - 1;
    __nv_bfloat16* out = last ? n->eb[l].v : n->cat[l].v;
    if ((e = fwd(n, n->conv[n->enc_b[l]], B, n->ea[l].v, n->ch[l], 0, out, last ? n->ch[l] : 2 * n->ch[l],
                 last ? 0 : n->ch[l], train)) != cudaSuccess)
      return e;
  }
  const __nv_bfloat16* din = n->eb[L - 1].v;
  for (int l = L - 2; l >= 0; --l) {
    const int c = n->ch[l], cu = n->ch[l + 1];
    if ((e = fwd(n, n->conv[n->up[l]], B, din, cu, 0, n->cat[l].v, 2 * c, 0, train, 1)) != cudaSuccess) return e;
    if ((e = fwd(n, n->conv[n->dec_a[l]], B, n->cat[l].v, 2 * c, 0, n->da[l].v, c, 0, train)) != cudaSuccess)
      return e;
    if ((e = fwd(n, n->conv[n->dec_b[l]], B, n->da[l].v, c, 0, n->db[l].v, c, 0, train)) != cudaSuccess) return e;
    din = n->db[l].v;
  }
  return head_fwd(din, n->ch[0], n->P + n->head_w, n->P + n->head_b, n->out, n->out_ch, npix_at(n, 0, B), x,
                  n->in_ch, n->norm, n->stream);
}

static cudaError_t backward(gpe2p_net* n, int B) {
  const int L = n->L;
  const __nv_bfloat16* din = L > 1 ? n->db[0].v : n->eb[0].v;
  __nv_bfloat16* gdin = L > 1 ? n->db[0].g : n->eb[0].g;
  cudaError_t e = head_bwd(din, n->ch[0], n->P + n->head_w, n->dout, n->out_ch, gdin, n->G + n->head_w,
                           n->G + n->head_b, npix_at(n, 0, B), n->stream);
  if (e != cudaSuccess) return e;
  // decoder, from the output up to the bottleneck
  for (int l = 0; l <= L - 2; ++l) {
    const int c = n->ch[l], cu = n->ch[l + 1];
    if ((e = bwd(n, n->conv[n->dec_b[l]], B, n->da[l].v, c, 0, n->db[l].g, c, 0, n->da[l].g, c, 0, 0)) != cudaSuccess)
      return e;
    if ((e = bwd(n, n->conv[n->dec_a[l]], B, n->cat[l].v, 2 * c, 0, n->da[l].g, c, 0, n->cat[l].g, 2 * c, 0, 0)) !=
        cudaSuccess)
      return e;
    if ((e = copy_ch(n->cat[l].g, 2 * c, c, n->eb[l].g, c, 0, npix_at(n, l, B), c, 0, n->stream)) != cudaSuccess)
      return e;
    const __nv_bfloat16* dlow = l + 1 <= L - 2 ? n->db[l + 1].v : n->eb[L - 1].v;
    if ((e = bwd(n, n->conv[n->up[l]], B, dlow, cu, 0, n->cat[l].g, 2 * c, 0, n->upx[l].g, cu, 0, 0, 1)) !=
        cudaSuccess)
      return e;
    __nv_bfloat16* gnext = l + 1 <= L - 2 ? n->db[l + 1].g : n->eb[L - 1].g;
    if ((e = up_bwd(n->upx[l].g, gnext, B, n->H >> l, n->W >> l, cu, n->stream)) != cudaSuccess) return e;
  }
  // encoder, from the bottleneck down
  for (int l = L - 1; l >= 0; --l) {
    const int c = n->ch[l];
    if ((e = bwd(n, n->conv[n->enc_b[l]], B, n->ea[l].v, c, 0, n->eb[l].g, c, 0, n->ea[l].g, c, 0, 0)) != cudaSuccess)
      return e;
    const __nv_bfloat16* in = l > 0 ? n->pooled[l - 1].v : n->in16.v;
    const int ldin = l > 0 ? n->ch[l - 1] : 16;
    __nv_bfloat16* gin = l > 0 ? n->pooled[l - 1].g : nullptr;
    if ((e = bwd(n, n->conv[n->enc_a[l]], B, in, ldin, 0, n->ea[l].g, c, 0, gin, ldin, 0, 0)) != cudaSuccess)
      return e;
    if (l > 0) {
      const int cp = n->ch[l - 1];
      if ((e = pool_bwd(n->pooled[l - 1].g, n->eb[l - 1].g, cp, 0, B, n->H >> (l - 1), n->W >> (l - 1), cp, 1,
                        n->stream)) != cudaSuccess)
        return e;
    }
  }
  return cudaSuccess;
}

extern "C" int gpe2p_net_create(int levels, const int* channels, int in_ch, int out_ch, int H, int W, int max_batch,
                                unsigned long long seed, void* stream, gpe2p_net_handle* out) {
  if (!out || !channels) return net_fail(nullptr, GPE2P_EINVAL, "NULL argument");
  *out = nullptr;
  if (levels < 1 || levels > 6) return net_fail(nullptr, GPE2P_EINVAL, "levels must lie in [1, 6]");
  if (in_ch < 1 || in_ch > 16 || out_ch < 1 || out_ch > 16)
    return net_fail(nullptr, GPE2P_EINVAL, "in and out channels must lie in [1, 16]");
  for (int l = 0; l < levels; ++l)
    if (channels[l] < 16 || channels[l] % 16 || channels[l] > 1024)
      return net_fail(nullptr, GPE2P_EINVAL, "channels must be multiples of 16 in [16, 1024]");
  const int div = 1 << (levels - 1);
  if (H < div || W < div || H % div || W % div)
    return net_fail(nullptr, GPE2P_EINVAL, "H and W must be multiples of 2^(levels-1)");
  if (max_batch < 1 || (long long)max_batch * H * W > (1LL << 31) / 64)
    return net_fail(nullptr, GPE2P_EINVAL, "max_batch * H * W too large");
  gpe2p_net* n = new (std::nothrow) gpe2p_net();
  if (!n) return net_fail(nullptr, GPE2P_ENOMEM, "host allocation failed");
  n->L = levels;
  n->ch.assign(channels, channels + levels);
  n->in_ch = in_ch;
  n->out_ch = out_ch;
  n->H = H;
  n->W = W;
  n->maxB = max_batch;
  for (int c = 0; c < 16; ++c) {
    n->norm.mean[c] = 0.f;
    n->norm.inv[c] = 1.f;
    n->norm.oscale[c] = 1.f;
  }
  n->norm.residual = 0;
  cudaError_t e = cudaSuccess;
  if (stream) n->stream = (cudaStream_t)stream;
  else {
    e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
    n->own_stream = true;
  }
  // layers
  n->enc_a.resize(levels);
  n->enc_b.resize(levels);
  n->up.assign(levels, -1);
  n->dec_a.assign(levels, -1);
  n->dec_b.assign(levels, -1);
  for (int l = 0; l < levels; ++l) {
    n->enc_a[l] = add_conv(n, l == 0 ? 16 : n->ch[l - 1], n->ch[l], 9, l);
    n->enc_b[l] = add_conv(n, n->ch[l], n->ch[l], 9, l);
  }
  for (int l = levels - 2; l >= 0; --l) {
    n->up[l] = add_conv(n, n->ch[l + 1], n->ch[l], 9, l);
    n->dec_a[l] = add_conv(n, 2 * n->ch[l], n->ch[l], 9, l);
    n->dec_b[l] = add_conv(n, n->ch[l], n->ch[l], 9, l);
  }
  n->head_w = n->nparam;
  n->nparam += (long long)out_ch * n->ch[0];
  n->head_b = n->nparam;
  n->nparam += out_ch;
  const int B = max_batch;
  auto fail_alloc = [&](cudaError_t ee) {
    gpe2p_net_destroy(n);
    return net_fail(nullptr, GPE2P_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(ee));
  };
  if (e != cudaSuccess) return fail_alloc(e);
  if ((e = nalloc(n, &n->P, n->nparam)) || (e = nalloc(n, &n->G, n->nparam)) || (e = nalloc(n, &n->Am, n->nparam)) ||
      (e = nalloc(n, &n->Av, n->nparam)))
    return fail_alloc(e);
  long long zmax = 0;
  for (auto& c : n->conv) {
    const long long np = npix_at(n, c.level, B);
    if (c.taps == 9 && ((e = nalloc(n, &c.wtp, (size_t)c.cout * c.taps * c.cin)) ||
                        (e = nalloc(n, &c.wdp, (size_t)c.cout * c.taps * c.cin))))
      return fail_alloc(e);
    if ((e = nalloc(n, &c.wt, (size_t)c.cout * c.taps * c.cin)) || (e = nalloc(n, &c.wd, (size_t)c.cout * c.taps * c.cin)) ||
        (e = nalloc(n, &c.z, (size_t)np * c.cout)))
      return fail_alloc(e);
    if (np * c.cout > zmax) zmax = np * c.cout;
  }
  auto mk = [&](Act& a, int c, int level) -> cudaError_t {
    a.c = c;
    a.level = level;
    const size_t cnt = (size_t)npix_at(n, level, B) * c;
    cudaError_t ee = nalloc(n, &a.v, cnt);
    if (ee == cudaSuccess) ee = nalloc(n, &a.g, cnt);
    return ee;
  };
  n->ea.resize(levels);
  n->eb.resize(levels);
  n->pooled.resize(levels);
  n->upx.resize(levels);
  n->cat.resize(levels);
  n->da.resize(levels);
  n->db.resize(levels);
  if ((e = mk(n->in16, 16, 0))) return fail_alloc(e);
  for (int l = 0; l < levels; ++l) {
    if ((e = mk(n->ea[l], n->ch[l], l)) || (e = mk(n->eb[l], n->ch[l], l))) return fail_alloc(e);
    if (l < levels - 1) {
      if ((e = mk(n->pooled[l], n->ch[l], l + 1)) || (e = mk(n->upx[l], n->ch[l + 1], l)) ||
          (e = mk(n->cat[l], 2 * n->ch[l], l)) || (e = mk(n->da[l], n->ch[l], l)) || (e = mk(n->db[l], n->ch[l], l)))
        return fail_alloc(e);
    }
  }
  if ((e = nalloc(n, &n->dz, (size_t)zmax)) || (e = nalloc(n, &n->out, (size_t)npix_at(n, 0, B) * out_ch)) ||
      (e = nalloc(n, &n->dout, (size_t)npix_at(n, 0, B) * out_ch)) || (e = nalloc(n, &n->loss, 1)) ||
      (e = nalloc(n, &n->d_err, 1)))
    return fail_alloc(e);
  if ((e = cudaMallocHost((void**)&n->loss_h, sizeof(float)))) return fail_alloc(e);
  if ((e = cudaMallocHost((void**)&n->h_err, sizeof(int)))) return fail_alloc(e);
  if ((e = cudaMemset(n->d_err, 0, sizeof(int)))) return fail_alloc(e);
  // He-uniform initial weights (seeded), zero biases, a small head
  std::vector<float> p(n->nparam, 0.f);
  std::mt19937_64 rng(seed);
  for (auto& c : n->conv) {
    const int fan_in = c.taps * (c.level == 0 && &c == &n->conv[n->enc_a[0]] ? in_ch : c.cin);
    const float lim = std::sqrt(6.0f / (float)fan_in);
    std::uniform_real_distribution<float> U(-lim, lim);
    for (long long i = 0; i < (long long)c.cout * c.taps * c.cin; ++i) p[c.w + i] = U(rng);
  }
  {
    const float lim = 0.01f * std::sqrt(6.0f / (float)n->ch[0]);
    std::uniform_real_distribution<float> U(-lim, lim);
    for (long long i = 0; i < (long long)out_ch * n->ch[0]; ++i) p[n->head_w + i] = U(rng);
  }
  if ((e = cudaMemcpy(n->P, p.data(), n->nparam * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(n->Am, 0, n->nparam * sizeof(float))) || (e = cudaMemset(n->Av, 0, n->nparam * sizeof(float))) ||
      (e = refresh_bf16(n)) || (e = cudaStreamSynchronize(n->stream))) {
    gpe2p_net_destroy(n);
    return net_fail(nullptr, GPE2P_ECUDA, std::string("net set-up: ") + cudaGetErrorString(e));
  }
  *out = n;
  return GPE2P_OK;
}

extern "C" int gpe2p_net_set_normalization(gpe2p_net_handle n, const float* in_mean, const float* in_scale,
                                           const float* out_scale, int residual) {
  if (!n) return net_fail(n, GPE2P_EINVAL, "NULL handle");
  if (residual != 0 && residual != 1) return net_fail(n, GPE2P_EINVAL, "residual must be 0 or 1");
  if (residual && n->out_ch > n->in_ch) return net_fail(n, GPE2P_EINVAL, "residual needs out_ch <= in_ch");
  Norm nm = n->norm;
  for (int c = 0; c < n->in_ch; ++c) {
    const float m = in_mean ? in_mean[c] : 0.f, s = in_scale ? in_scale[c] : 1.f;
    if (!std::isfinite(m) || !std::isfinite(s) || !(s != 0.f)) return net_fail(n, GPE2P_EINVAL, "bad input normalisation");
    nm.mean[c] = m;
    nm.inv[c] = 1.0f / s;
  }
  for (int c = 0; c < n->out_ch; ++c) {
    const float s = out_scale ? out_scale[c] : 1.f;
    if (!std::isfinite(s) || !(s != 0.f)) return net_fail(n, GPE2P_EINVAL, "bad output scale");
    nm.oscale[c] = s;
  }
  nm.residual = residual;
  n->norm = nm;
  drop_forward_graph(n);
  return GPE2P_OK;
}

// after a synchronisation: GPE2P_ETIMEOUT if a tcgen05 kernel gave up a wait
static int net_err_word(gpe2p_net* n) {
  NK(n, cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream), "error word");
  NK(n, cudaStreamSynchronize(n->stream), "error word");
  if (*n->h_err) return net_fail(n, GPE2P_ETIMEOUT, "a tensor-core kernel timed out waiting for its MMAs");
  return GPE2P_OK;
}

extern "C" int gpe2p_net_sync(gpe2p_net_handle n) {
  if (!n) return net_fail(n, GPE2P_EINVAL, "NULL handle");
  return net_err_word(n);
}

extern "C" int gpe2p_net_fault(gpe2p_net_handle n, int what, int value) {
  if (!n) return net_fail(n, GPE2P_EINVAL, "NULL handle");
  if (what == GPE2P_FAULT_LOSE_COPY) {
    if (value != 0 && value != 1) return net_fail(n, GPE2P_EINVAL, "bad fault value");
    n->wait_fault = value;
  } else if (what == GPE2P_FAULT_CLEAR) {
    n->wait_fault = 0;
    NK(n, cudaStreamSynchronize(n->stream), "fault clear");
    NK(n, cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream), "fault clear");
    NK(n, cudaStreamSynchronize(n->stream), "fault clear");
  } else {
    return net_fail(n, GPE2P_EINVAL, "fault kind not taken by a network");
  }
  drop_forward_graph(n);
  return GPE2P_OK;
}

extern "C" int gpe2p_net_set_backend(gpe2p_net_handle n, int tcgen05) {
  if (!n || (tcgen05 != 0 && tcgen05 != 1)) return net_fail(n, GPE2P_EINVAL, "bad arguments");
  n->use_tc = tcgen05;
  drop_forward_graph(n);
  return GPE2P_OK;
}

extern "C" long long gpe2p_net_num_params(gpe2p_net_handle n) { return n ? n->nparam : -1; }

extern "C" int gpe2p_net_get_params(gpe2p_net_handle n, float* host, long long count) {
  if (!n || !host || count != n->nparam) return net_fail(n, GPE2P_EINVAL, "bad arguments");
  NK(n, cudaMemcpyAsync(host, n->P, count * sizeof(float), cudaMemcpyDeviceToHost, n->stream), "get params");
  NK(n, cudaStreamSynchronize(n->stream), "get params");
  return GPE2P_OK;
}

extern "C" int gpe2p_net_set_params(gpe2p_net_handle n, const float* host, long long count) {
  if (!n || !host || count != n->nparam) return net_fail(n, GPE2P_EINVAL, "bad arguments");
  NK(n, cudaMemcpyAsync(n->P, host, count * sizeof(float), cudaMemcpyHostToDevice, n->stream), "set params");
  NK(n, refresh_bf16(n), "set params");
  NK(n, cudaMemsetAsync(n->Am, 0, count * sizeof(float), n->stream), "set params");
  NK(n, cudaMemsetAsync(n->Av, 0, count * sizeof(float), n->stream), "set params");
  n->adam_t = 0;
  NK(n, cudaStreamSynchronize(n->stream), "set params");
  return GPE2P_OK;
}

static void drop_forward_graph(gpe2p_net* n) {
  if (n->fwd_exec) cudaGraphExecDestroy(n->fwd_exec);
  n->fwd_exec = nullptr;
  n->fwd_x = nullptr;
  n->fwd_y = nullptr;
  n->fwd_b = 0;
}

static cudaError_t enqueue_forward(gpe2p_net* n, const float* x, float* y, int batch) {
  cudaError_t e = forward(n, x, batch, false);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(y, n->out, (size_t)npix_at(n, 0, batch) * n->out_ch * sizeof(float),
                         cudaMemcpyDeviceToDevice, n->stream);
}

// The forward of a given (x, y, batch) is captured once into a CUDA graph and
// replayed by later calls with the same arguments (the weights are read from
// device memory, so training between calls needs no new capture).
extern "C" int gpe2p_net_forward(gpe2p_net_handle n, const float* x, float* y, int batch) {
  if (!n || !x || !y || batch < 1 || batch > n->maxB) return net_fail(n, GPE2P_EINVAL, "bad arguments");
  if (!(n->fwd_exec && n->fwd_x == x && n->fwd_y == y && n->fwd_b == batch)) {
    drop_forward_graph(n);
    cudaGraph_t g = nullptr;
    NK(n, cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeRelaxed), "forward capture");
    const cudaError_t e = enqueue_forward(n, x, y, batch);
    const cudaError_t e2 = cudaStreamEndCapture(n->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      NK(n, e != cudaSuccess ? e : e2, "forward capture");
    }
    const cudaError_t e3 = cudaGraphInstantiate(&n->fwd_exec, g, 0);
    cudaGraphDestroy(g);
    NK(n, e3, "forward graph");
    n->fwd_x = x;
    n->fwd_y = y;
    n->fwd_b = batch;
  }
  NK(n, cudaGraphLaunch(n->fwd_exec, n->stream), "forward");
  return GPE2P_OK;
}

static int loss_and_grads(gpe2p_net* n, const float* x, const float* t, int batch) {
  NK(n, cudaMemsetAsync(n->G, 0, n->nparam * sizeof(float), n->stream), "zero grads");
  NK(n, cudaMemsetAsync(n->loss, 0, sizeof(float), n->stream), "zero loss");
  NK(n, forward(n, x, batch, true), "forward");
  NK(n, mse(n->out, t, n->dout, npix_at(n, 0, batch) * n->out_ch, n->out_ch, n->norm, n->loss, n->stream), "loss");
  NK(n, backward(n, batch), "backward");
  return GPE2P_OK;
}

extern "C" int gpe2p_net_gradients(gpe2p_net_handle n, const float* x, const float* t, int batch, float* grad,
                                   float* loss) {
  if (!n || !x || !t || batch < 1 || batch > n->maxB) return net_fail(n, GPE2P_EINVAL, "bad arguments");
  int rc = loss_and_grads(n, x, t, batch);
  if (rc != GPE2P_OK) return rc;
  if (grad) NK(n, cudaMemcpyAsync(grad, n->G, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream), "grads");
  NK(n, cudaMemcpyAsync(n->loss_h, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream), "loss");
  NK(n, cudaStreamSynchronize(n->stream), "gradients");
  if (loss) *loss = *n->loss_h;
  return net_err_word(n);
}

extern "C" int gpe2p_net_train_step(gpe2p_net_handle n, const float* x, const float* t, int batch, float lr,
                                    float* loss) {
  if (!n || !x || !t || batch < 1 || batch > n->maxB || !(lr >= 0.f))
    return net_fail(n, GPE2P_EINVAL, "bad arguments");
  int rc = loss_and_grads(n, x, t, batch);
  if (rc != GPE2P_OK) return rc;
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)n->adam_t), c2 = 1.0f - std::pow(b2, (float)n->adam_t);
  NK(n, adam(n->P, n->G, n->Am, n->Av, n->nparam, lr, b1, b2, 1e-8f, c1, c2, n->stream), "adam");
  NK(n, refresh_bf16(n), "weights");
  if (loss) {
    NK(n, cudaMemcpyAsync(n->loss_h, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream), "loss");
    NK(n, cudaStreamSynchronize(n->stream), "train step");
    *loss = *n->loss_h;
    return net_err_word(n);
  }
  return GPE2P_OK;
}

extern "C" double gpe2p_net_flops(gpe2p_net_handle n, int batch) {
  if (!n) return 0.0;
  double f = 0.0;
  for (auto& c : n->conv) f += 2.0 * (double)npix_at(n, c.level, batch) * c.cout * c.taps * c.cin;
  f += 2.0 * (double)npix_at(n, 0, batch) * n->out_ch * n->ch[0];
  return f;
}

extern "C" const char* gpe2p_net_last_error(gpe2p_net_handle n) { return n ? n->err.c_str() : g_net_error.c_str(); }

extern "C" void gpe2p_net_destroy(gpe2p_net_handle n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  drop_forward_graph(n);
  for (void* p : n->allocs) cudaFree(p);
  if (n->loss_h) cudaFreeHost(n->loss_h);
  if (n->h_err) cudaFreeHost(n->h_err);
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
}
