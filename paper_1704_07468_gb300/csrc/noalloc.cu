// Gram kernel of one dataset without any memory allocation.
//
// Some callers cannot let a library allocate device memory: applications
// whose GPU memory is owned by a framework's caching allocator or carved
// into fixed budgets up front (a stray cudaMalloc fragments the pool or
// breaks the budget), latency-sensitive request paths where cudaMalloc and
// cudaFree would synchronise the whole device, and plug-ins that are handed
// input and output buffers but are not allowed to own device memory.  For
// them, gakco_gram_device_noalloc runs the per-mask pipeline (pack, sort and
// run-length count per mask, countAndUpdate into C_m, inclusion-exclusion,
// kernel, normalisation) with every intermediate buffer carved out of one
// file-scope static device array, and every host-side table staged in one
// file-scope static host array.  It calls no cudaMalloc, cudaFree,
// cudaMallocHost or other allocating routine, and creates no stream or event.
//
// The static device array (kScratchBytes) is part of the library image: each
// GPU that loads the library holds it until the process exits.  All calls
// share it and it keeps the previous call's contents; everything that must
// start at zero is cleared at the start of each call.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "gakco.h"
#include "launch.h"

using namespace gk;

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;     // device scratch, 64 MiB
constexpr size_t kHostTableBytes = (size_t)1 << 20;    // host staging, 1 MiB
constexpr int kMaxMasks = 1024;                        // c_gk limit of this entry
constexpr int kMaxDevices = 64;
constexpr int kRadixBits = 8;                          // sort digit width

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host copies of the table area; reused by every call on every device, so
// calls hold g_lock (a plain mutex, which allocates nothing) from start to
// finish.
static std::mutex g_lock;
static unsigned char h_tables[kHostTableBytes];
static MaskDesc h_masks[kMaxMasks];
static uint32_t h_level[kMaxMasks];

// Device address of g_scratch per device.  It is looked up again (with the
// kernel attributes set again) on every call made outside stream capture,
// so a device reset or a new primary context, which reloads the module,
// leaves no stale address behind; a call made while `stream` is capturing
// uses the address of the last call outside capture.
static unsigned char* d_scratch[kMaxDevices];
static bool d_ready[kMaxDevices];

int set_err(char* err, int len, int code, const char* msg) {
  if (err && len > 0) snprintf(err, (size_t)len, "%s", msg);
  return code;
}

uint64_t binom(int n, int r) {
  if (r < 0 || r > n) return 0;
  uint64_t v = 1;
  for (int i = 1; i <= r; ++i) v = v * (uint64_t)(n - r + i) / (uint64_t)i;
  return v;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }
size_t up16(size_t v) { return (v + 15) / 16 * 16; }

// Position masks in level order (deleted sets in lexicographic order within
// a level), as in the main engine.  Returns the mask count.
int make_masks(int g, int M, int bits) {
  int cnt = 0;
  for (int m = 0; m <= M; ++m) {
    int del[kMaxLevels] = {};
    for (int i = 0; i < m; ++i) del[i] = i;
    for (;;) {
      int keep[64], nk = 0;
      for (int q = 0, j = 0; q < g; ++q) {
        if (j < m && del[j] == q)
          ++j;
        else
          keep[nk++] = q;
      }
      MaskDesc md{};
      md.level = (uint32_t)m;
      md.kbits = (uint32_t)((g - m) * bits);
      for (int i = 0; i < nk;) {
        int j = i;
        while (j + 1 < nk && keep[j + 1] == keep[j] + 1) ++j;
        const int len = j - i + 1;
        md.sr[md.nruns] = (uint32_t)(bits * (g - 1 - keep[j]));
        md.sl[md.nruns] = (uint32_t)(bits * (nk - 1 - j));
        md.msk[md.nruns] = len * bits >= 64 ? ~0ull : ((1ull << (len * bits)) - 1);
        md.nruns++;
        i = j + 1;
      }
      h_masks[cnt] = md;
      h_level[cnt] = (uint32_t)m;
      ++cnt;
      int i = m - 1;
      while (i >= 0 && del[i] == g - m + i) --i;
      if (i < 0) break;
      del[i]++;
      for (int j = i + 1; j < m; ++j) del[j] = del[j - 1] + 1;
    }
  }
  return cnt;
}

}  // namespace

extern "C" int gakco_gram_device_noalloc(int sigma, int g, int k, const uint8_t* codes,
                                         const int64_t* offsets, int32_t n, int32_t* K,
                                         double* Khat, int32_t* Nm, void* stream_v, char* err,
                                         int err_len) {
  char msg[256];
  if (err && err_len > 0) err[0] = '\0';
  // --- parameters -------------------------------------------------------
  if (sigma < 2 || sigma > 255 || g < 1 || k < 1 || k > g)
    return set_err(err, err_len, GAKCO_E_INVALID, "need 2 <= sigma <= 255 and 1 <= k <= g");
  int bits = 0;
  while ((1 << bits) < sigma) ++bits;
  const int M = g - k;
  if (g * bits > 64 || M + 1 > kMaxLevels)
    return set_err(err, err_len, GAKCO_E_INVALID, "g * ceil(log2 sigma) must be <= 64 and g - k <= 15");
  uint64_t cgk = 0;
  uint32_t maxC = 0;
  for (int m = 0; m <= M; ++m) {
    cgk += binom(g, m);
    if (binom(g, m) > maxC) maxC = (uint32_t)binom(g, m);
  }
  if (cgk > (uint64_t)kMaxMasks) {
    snprintf(msg, sizeof msg, "%llu position masks; this entry point handles at most %d",
             (unsigned long long)cgk, kMaxMasks);
    return set_err(err, err_len, GAKCO_E_OVERFLOW, msg);
  }
  if (n < 0 || n > 65535) return set_err(err, err_len, GAKCO_E_INVALID, "n must be in [0, 65535]");
  if (n > 0 && (!offsets || !K)) return set_err(err, err_len, GAKCO_E_INVALID, "offsets and K are required");
  if (n == 0) return GAKCO_OK;

  // --- dataset: windows and the int32 bound ---------------------------------
  uint64_t G = 0, wmax = 0;
  for (int32_t x = 0; x < n; ++x) {
    const int64_t len = offsets[x + 1] - offsets[x];
    if (offsets[x] < 0 || len < 0)
      return set_err(err, err_len, GAKCO_E_INVALID, "offsets must be non-negative and non-decreasing");
    const uint64_t W = len >= g ? (uint64_t)(len - g + 1) : 0;
    if (W > 65535) return set_err(err, err_len, GAKCO_E_OVERFLOW, "a sequence has more than 65535 windows");
    if (W > wmax) wmax = W;
    G += W;
  }
  if (offsets[n] > 0 && !codes) return set_err(err, err_len, GAKCO_E_INVALID, "codes is null");
  if ((long double)maxC * (long double)wmax * (long double)wmax >= 2147483648.0L)
    return set_err(err, err_len, GAKCO_E_OVERFLOW, "C(g,m) * W_max^2 reaches 2^31; int32 kernel would overflow");
  if (G >= 0xFFFFFFFFull) return set_err(err, err_len, GAKCO_E_OVERFLOW, "2^32 or more windows");

  // --- scratch layout (device) ----------------------------------------------
  const bool wide = g * bits > 32;
  const size_t kb = wide ? 8 : 4;
  const uint32_t ntiles = (uint32_t)((G + kTile - 1) / kTile);
  const size_t nn = (size_t)n * (size_t)n;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = up256(o + bytes);
    return r;
  };
  // Host-built table area, copied as one block.
  size_t t = 0;
  auto ttake = [&](size_t bytes) {
    const size_t r = t;
    t = up16(t + bytes);
    return r;
  };
  const size_t t_masks = ttake(cgk * sizeof(MaskDesc));
  const size_t t_segs = ttake(cgk * sizeof(SegDesc));
  const size_t t_tiles = ttake((size_t)ntiles * 4 + 4);
  const size_t t_coff = ttake((size_t)(n + 1) * 8);
  const size_t t_woff = ttake((size_t)(n + 1) * 4);
  const size_t t_pack = ttake(sizeof(DsPack));
  const size_t t_info = ttake(sizeof(DsInfo));
  if (t > kHostTableBytes)
    return set_err(err, err_len, GAKCO_E_OVERFLOW, "input too large for this entry point's table area (1 MiB)");
  const size_t o_tables = take(t);
  const size_t o_fullkey = take(G * 8);
  const size_t o_wid = take(G * 4);
  const size_t o_ewin = take(G * 4);
  const size_t o_eseq = take(G * 4);
  const size_t o_efe = take(G * 4);
  const size_t o_keyA = take(G * kb);
  const size_t o_keyB = take(G * kb);
  const size_t o_valA = take(G * 4);
  const size_t o_valB = take(G * 4);
  const size_t o_hist = take(((size_t)1 << kRadixBits) * ntiles * 4);
  const size_t o_dtot = take(((size_t)1 << kRadixBits) * 4);
  const size_t o_tcnt = take((size_t)ntiles * 8);
  const size_t o_segtot = take(64);
  const size_t o_estart = take((G + 2) * 4);
  const size_t o_etseq = take((G + 2) * 4);
  const size_t o_efid = take((G + 2) * 4);
  const size_t o_fstart = take((G + 2) * 4);
  const size_t o_C = take((size_t)(M + 1) * nn * 4);
  const size_t o_rinv = take((size_t)n * 8);
  const size_t o_status = take(128);
  if (o > kScratchBytes) {
    snprintf(msg, sizeof msg,
             "input needs %zu bytes of scratch; the static scratch area holds %zu (64 MiB)", o,
             kScratchBytes);
    return set_err(err, err_len, GAKCO_E_OVERFLOW, msg);
  }

  // --- per-device set-up: device address of the static array ---------------
  std::lock_guard<std::mutex> hold(g_lock);
  cudaStream_t st = (cudaStream_t)stream_v;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_err(err, err_len, GAKCO_E_CUDA, "no usable CUDA device");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(msg, sizeof msg, "stream query: %s", cudaGetErrorString(e));
    return set_err(err, err_len, GAKCO_E_CUDA, msg);
  }
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      return set_err(err, err_len, GAKCO_E_CUDA, msg);
    }
    e = (cudaError_t)prep_init();  // kernel attributes (shared-memory limits); no allocation
    if (e != cudaSuccess) {
      cudaGetLastError();
      snprintf(msg, sizeof msg, "kernel attribute set-up: %s", cudaGetErrorString(e));
      return set_err(err, err_len, GAKCO_E_CUDA, msg);
    }
    d_scratch[dev] = (unsigned char*)p;
    d_ready[dev] = true;
  } else if (!d_ready[dev]) {
    return set_err(err, err_len, GAKCO_E_INVALID,
                   "first call on this device made during stream capture; call once outside capture first");
  }
  unsigned char* S = d_scratch[dev];

  // --- host tables -----------------------------------------------------------
  const int nm = make_masks(g, M, bits);
  memcpy(h_tables + t_masks, h_masks, (size_t)nm * sizeof(MaskDesc));
  SegDesc* segs = (SegDesc*)(h_tables + t_segs);
  for (int mu = 0; mu < nm; ++mu) {
    SegDesc s{};
    s.base = 0;      // one segment per launch: chunk-local offsets start at 0
    s.pool = 0;      // one mask's entries at a time
    s.hist = 0;
    s.G = (uint32_t)G;
    s.win0 = 0;
    s.mask = (uint32_t)mu;
    s.tile0 = 0;
    s.ntiles = ntiles;
    s.ds = 0;
    segs[mu] = s;
  }
  memset(h_tables + t_tiles, 0, (size_t)ntiles * 4 + 4);  // every tile is segment 0
  memcpy(h_tables + t_coff, offsets, (size_t)(n + 1) * 8);
  uint32_t* woff = (uint32_t*)(h_tables + t_woff);
  woff[0] = 0;
  for (int32_t x = 0; x < n; ++x) {
    const int64_t len = offsets[x + 1] - offsets[x];
    woff[x + 1] = woff[x] + (uint32_t)(len >= g ? len - g + 1 : 0);
  }
  DsPack pk{};
  pk.codes = codes;
  pk.coff = (const int64_t*)(S + o_tables + t_coff);
  pk.woff = (const uint32_t*)(S + o_tables + t_woff);
  pk.win0 = 0;
  pk.n = (uint32_t)n;
  pk.seq0 = 0;
  memcpy(h_tables + t_pack, &pk, sizeof pk);
  DsInfo in{};
  in.woff = pk.woff;
  in.K = K;
  in.Nm = Nm;
  in.Khat = Khat;
  in.rinv = (double*)(S + o_rinv);
  in.win0 = 0;
  in.n = (uint32_t)n;
  in.tile0 = 0;
  memcpy(h_tables + t_info, &in, sizeof in);
  AccParams coef{};
  coef.M = (uint32_t)M;
  coef.status = (uint32_t*)(S + o_status);
  for (int m = 0; m <= M; ++m) {
    coef.h[m] = (uint32_t)binom(g - m, k);
    for (int j = 0; j < m; ++j) coef.ie[m][j] = (uint32_t)binom(g - j, m - j);
  }

  // --- work on the caller's stream -------------------------------------------
  // From pageable memory the copy is staged before the call returns, so the
  // static host table area may be rewritten by the next call.
  e = cudaMemcpyAsync(S + o_tables, h_tables, t, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S + o_status, 0, 128, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S + o_C, 0, (size_t)(M + 1) * nn * 4, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(msg, sizeof msg, "staging: %s", cudaGetErrorString(e));
    return set_err(err, err_len, GAKCO_E_CUDA, msg);
  }
  uint32_t* status = (uint32_t*)(S + o_status);
  launch_pack((const DsPack*)(S + o_tables + t_pack), 1, (uint32_t)n, g, bits, sigma,
              (uint64_t*)(S + o_fullkey), (uint32_t*)(S + o_wid), status, st);
  const SegDesc* d_segs = (const SegDesc*)(S + o_tables + t_segs);
  const uint32_t* d_tiles = (const uint32_t*)(S + o_tables + t_tiles);
  const MaskDesc* d_masks = (const MaskDesc*)(S + o_tables + t_masks);
  if (G > 0) {
    for (int mu = 0; mu < nm; ++mu) {
      const int m = (int)h_level[mu];
      const int kbits = (g - m) * bits;
      const int np = (kbits + kRadixBits - 1) / kRadixBits;
      const int rb = (kbits + np - 1) / np;
      const bool w = kbits > 32;
      void* kbuf[2] = {S + o_keyA, S + o_keyB};
      uint32_t* vbuf[2] = {(uint32_t*)(S + o_valA), (uint32_t*)(S + o_valB)};
      void* kin = kbuf[1];  // the first pass extracts the masked keys here
      const uint32_t* vin = (const uint32_t*)(S + o_wid);  // first-pass payload: window ids
      int cur = 0;
      for (int q = 0; q < np; ++q) {
        const int shift = q * rb;
        const int nb = rb < kbits - shift ? rb : kbits - shift;
        launch_sort_pass(w, q == 0, d_segs + mu, 1, d_tiles, ntiles, d_masks,
                         (const uint64_t*)(S + o_fullkey), kin, vin, kbuf[cur], vbuf[cur],
                         (uint32_t*)(S + o_hist), (uint32_t*)(S + o_dtot), shift, nb, st);
        kin = kbuf[cur];
        vin = vbuf[cur];
        cur ^= 1;
      }
      launch_rle(w, d_segs + mu, 1, d_tiles, ntiles, kin, vin, (const DsPack*)(S + o_tables + t_pack),
                 (uint32_t*)(S + o_tcnt), (uint32_t*)(S + o_segtot), (uint32_t*)(S + o_estart),
                 (uint32_t*)(S + o_etseq), (uint32_t*)(S + o_efid), (uint32_t*)(S + o_fstart),
                 (uint32_t*)(S + o_ewin), (uint32_t*)(S + o_eseq), (uint32_t*)(S + o_efe), st);
      launch_pairs_global((const uint32_t*)(S + o_segtot), (const uint32_t*)(S + o_eseq),
                          (const uint32_t*)(S + o_efe), (uint32_t)G,
                          (uint32_t*)(S + o_C) + (size_t)m * nn, (uint32_t)n, status, st);
    }
  }
  const DsInfo* d_info = (const DsInfo*)(S + o_tables + t_info);
  launch_ie_combine(d_info, (const uint32_t*)(S + o_C), (uint32_t)n, coef, st);
  const uint32_t nt = (uint32_t)((n + 31) / 32);
  launch_finish(d_info, 1, nt * nt, (uint32_t)M, Nm != nullptr, Khat != nullptr, st);
  e = cudaGetLastError();
  uint32_t hst[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst, status, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(msg, sizeof msg, "engine run: %s", cudaGetErrorString(e));
    return set_err(err, err_len, GAKCO_E_CUDA, msg);
  }
  if (hst[0] & kErrBadCode) return set_err(err, err_len, GAKCO_E_INVALID, "input holds a symbol >= sigma");
  if (hst[0]) {
    snprintf(msg, sizeof msg, "internal check failed (device status 0x%x)", hst[0]);
    return set_err(err, err_len, GAKCO_E_INTERNAL, msg);
  }
  return GAKCO_OK;
}
