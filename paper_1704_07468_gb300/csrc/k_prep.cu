// Preprocessing kernels: g-mer packing (Section 2.2, step 1), deletion of
// the masked positions (step 3), the lexicographic sort of the (g-m)-mers
// (steps 1 and 4; the "non-swapping" radix sort of Section S:1.2) and the
// counting of equal runs (step 2, countAndUpdate's counting half).
//
// The sort is a stable least-significant-digit radix sort over the masked
// key bits only.  Windows enter in (sequence, position) order, so stability
// leaves every run of equal keys ordered by sequence: no sequence bits need
// sorting.  Every launch covers all segments of a chunk, a segment being
// one (dataset, mask) pair, so one launch replaces hundreds of per-mask
// launches.
#include <cstdint>

#include "common.cuh"
#include "launch.h"

namespace gk {

namespace {

constexpr int kWarps = kSortThreads / 32;

// ---------------------------------------------------------------- packing --

// One block per sequence.  Writes the full g-mer key of every window (first
// symbol in the most significant bits, b bits per symbol) and the sequence
// index of every window.  Symbols >= sigma raise kErrBadCode.
__global__ void __launch_bounds__(128)
k_pack(const DsPack* __restrict__ ds, uint32_t nds, int g, int bits,
       int sigma, uint64_t* __restrict__ fullkey,
       uint32_t* __restrict__ win2seq, uint32_t* __restrict__ status) {
  const uint32_t gs = blockIdx.x;
  uint32_t d = 0;
  while (d + 1 < nds && ds[d + 1].seq0 <= gs) ++d;
  const DsPack D = ds[d];
  const uint32_t x = gs - D.seq0;
  const int64_t c0 = D.coff[x];
  const int64_t len = D.coff[x + 1] - c0;
  const uint8_t* __restrict__ s = D.codes + c0;
  // Validate every symbol of the sequence (also those no window covers).
  bool bad = false;
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x)
    bad |= s[i] >= sigma;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kErrBadCode);
  const uint32_t w0 = D.woff[x];
  const uint32_t W = D.woff[x + 1] - w0;
  const uint64_t base = D.win0 + w0;
  for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) {
    uint64_t key = 0;
    for (int p = 0; p < g; ++p) key = (key << bits) | s[i + p];
    fullkey[base + i] = key;
    win2seq[base + i] = x;
  }
}

// ------------------------------------------------------------ block scan --

// Exclusive scan of one value per thread across a kSortThreads block.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v,
                                                    uint32_t* sh_warp,
                                                    uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh_warp[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < kWarps ? sh_warp[lane] : 0;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    if (lane < kWarps) sh_warp[lane] = si - s;
    if (lane == kWarps - 1) sh_warp[kWarps] = si;
  }
  __syncthreads();
  uint32_t r = sh_warp[w] + incl - v;
  if (total) *total = sh_warp[kWarps];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------- radix sort --

template <typename KeyT, bool kFirst>
__device__ __forceinline__ KeyT load_key(const SegDesc& sd, uint64_t i,
                                         const MaskDesc& md,
                                         const uint64_t* __restrict__ fullkey,
                                         const KeyT* __restrict__ kin) {
  if (kFirst) return (KeyT)masked_key(fullkey[sd.win0 + i], md);
  return kin[sd.base + i];
}

// Per-tile digit counts: hist[seg.hist + digit * ntiles + tile].
template <typename KeyT, bool kFirst>
__global__ void __launch_bounds__(kSortThreads)
k_upsweep(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
          const MaskDesc* __restrict__ masks, const uint64_t* __restrict__ fullkey,
          const KeyT* __restrict__ kin, uint32_t* __restrict__ hist, int shift,
          int rbits) {
  extern __shared__ uint32_t sh[];
  __shared__ MaskDesc md;
  const uint32_t t = blockIdx.x;
  const SegDesc sd = segs[tile_seg[t]];
  const uint32_t lt = t - sd.tile0;
  const uint32_t radix = 1u << rbits;
  if (kFirst && threadIdx.x == 0) md = masks[sd.mask];
  for (uint32_t i = threadIdx.x; i < radix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    KeyT key = load_key<KeyT, kFirst>(sd, beg + i, md, fullkey, kin);
    atomicAdd(&sh[(uint32_t)(key >> shift) & (radix - 1)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < radix; i += blockDim.x)
    hist[sd.hist + (uint64_t)i * sd.ntiles + lt] = sh[i];
}

// Exclusive scan of each segment's digit-major counters, in place.
__global__ void __launch_bounds__(kSortThreads)
k_seg_scan(const SegDesc* __restrict__ segs, uint32_t* __restrict__ hist,
           int rbits) {
  __shared__ uint32_t sw[kWarps + 1];
  const SegDesc sd = segs[blockIdx.x];
  const uint64_t len = ((uint64_t)1 << rbits) * sd.ntiles;
  uint32_t* __restrict__ h = hist + sd.hist;
  uint32_t carry = 0;
  for (uint64_t b = 0; b < len; b += (uint64_t)kSortThreads * 4) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint64_t i = b + (uint64_t)threadIdx.x * 4 + q;
      v[q] = i < len ? h[i] : 0;
      s += v[q];
    }
    uint32_t tot;
    uint32_t pre = block_excl_scan(s, sw, &tot) + carry;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint64_t i = b + (uint64_t)threadIdx.x * 4 + q;
      if (i < len) h[i] = pre;
      pre += v[q];
    }
    carry += tot;
  }
}

// Stable scatter.  Warp w of the block owns elements
// [w*32*IPT, (w+1)*32*IPT) of the tile and visits them as j*32 + lane, so
// the visiting order is the element order; peers with the same digit are
// ranked with match.any, and running per-warp digit counts carry the rank
// across j.
template <typename KeyT, bool kFirst>
__global__ void __launch_bounds__(kSortThreads)
k_downsweep(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
            const MaskDesc* __restrict__ masks, const uint64_t* __restrict__ fullkey,
            const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin,
            KeyT* __restrict__ kout, uint32_t* __restrict__ vout,
            const uint32_t* __restrict__ hist, int shift, int rbits) {
  extern __shared__ uint32_t sh[];
  __shared__ MaskDesc md;
  const uint32_t radix = 1u << rbits;
  uint32_t* wc = sh;                   // kWarps x radix running counts
  uint32_t* gb = sh + kWarps * radix;  // radix global bases of this tile
  const uint32_t t = blockIdx.x;
  const SegDesc sd = segs[tile_seg[t]];
  const uint32_t lt = t - sd.tile0;
  if (kFirst && threadIdx.x == 0) md = masks[sd.mask];
  for (uint32_t i = threadIdx.x; i < kWarps * radix; i += blockDim.x) wc[i] = 0;
  for (uint32_t i = threadIdx.x; i < radix; i += blockDim.x)
    gb[i] = hist[sd.hist + (uint64_t)i * sd.ntiles + lt];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  const uint32_t lt_mask = lanemask_lt();
  KeyT keys[kSortIpt];
  uint32_t vals[kSortIpt];
  uint32_t rk[kSortIpt];
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    const bool valid = idx < cnt;
    KeyT key = 0;
    uint32_t val = 0;
    if (valid) {
      key = load_key<KeyT, kFirst>(sd, beg + idx, md, fullkey, kin);
      val = kFirst ? (uint32_t)(beg + idx) : vin[sd.base + beg + idx];
    }
    const uint32_t dg = valid ? ((uint32_t)(key >> shift) & (radix - 1)) : radix;
    const uint32_t peers = __match_any_sync(0xffffffffu, dg);
    const uint32_t rank = __popc(peers & lt_mask);
    const uint32_t base = valid ? wc[w * radix + dg] : 0;
    __syncwarp();
    if (valid && rank == 0) wc[w * radix + dg] = base + __popc(peers);
    __syncwarp();
    keys[j] = key;
    vals[j] = val;
    rk[j] = base + rank;
  }
  __syncthreads();
  for (uint32_t dg = threadIdx.x; dg < radix; dg += blockDim.x) {
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      uint32_t c = wc[ww * radix + dg];
      wc[ww * radix + dg] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    if (idx < cnt) {
      const uint32_t dg = (uint32_t)(keys[j] >> shift) & (radix - 1);
      const uint64_t pos = sd.base + gb[dg] + wc[w * radix + dg] + rk[j];
      kout[pos] = keys[j];
      vout[pos] = vals[j];
    }
  }
}

// ------------------------------------------------------------ run-length --

// Flags of sorted element i: a new entry starts where the (key, sequence)
// pair changes, a new feature where the key changes.
template <typename KeyT>
__device__ __forceinline__ void rle_flags(const SegDesc& sd, uint32_t i,
                                          const KeyT* __restrict__ keys,
                                          const uint32_t* __restrict__ vals,
                                          const uint32_t* __restrict__ win2seq,
                                          uint32_t& seq, bool& ne, bool& nf) {
  const KeyT k = keys[sd.base + i];
  seq = win2seq[sd.win0 + vals[sd.base + i]];
  if (i == 0) {
    ne = nf = true;
    return;
  }
  const KeyT kp = keys[sd.base + i - 1];
  const uint32_t sp = win2seq[sd.win0 + vals[sd.base + i - 1]];
  nf = k != kp;
  ne = nf || seq != sp;
}

template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads)
k_rle_count(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
            const KeyT* __restrict__ keys, const uint32_t* __restrict__ vals,
            const uint32_t* __restrict__ win2seq, uint32_t* __restrict__ tcnt) {
  __shared__ uint32_t sw[2][kWarps];
  const uint32_t t = blockIdx.x;
  const SegDesc sd = segs[tile_seg[t]];
  const uint32_t lt = t - sd.tile0;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  uint32_t ce = 0, cf = 0;
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    uint32_t seq;
    bool ne, nf;
    rle_flags<KeyT>(sd, (uint32_t)(beg + i), keys, vals, win2seq, seq, ne, nf);
    ce += ne;
    cf += nf;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ce += __shfl_xor_sync(0xffffffffu, ce, o);
    cf += __shfl_xor_sync(0xffffffffu, cf, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sw[0][w] = ce;
    sw[1][w] = cf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int i = 0; i < kWarps; ++i) {
      a += sw[0][i];
      b += sw[1][i];
    }
    tcnt[2 * (uint64_t)t] = a;
    tcnt[2 * (uint64_t)t + 1] = b;
  }
}

// Exclusive scan of the (entries, features) counts of each segment's tiles;
// totals go to segtot[2 * s] (E) and segtot[2 * s + 1] (F).
__global__ void __launch_bounds__(kSortThreads)
k_rle_scan(const SegDesc* __restrict__ segs, uint32_t* __restrict__ tcnt,
           uint32_t* __restrict__ segtot) {
  __shared__ uint32_t sw[kWarps + 1];
  const uint32_t s = blockIdx.x;
  const SegDesc sd = segs[s];
  uint32_t carry_e = 0, carry_f = 0;
  for (uint32_t b = 0; b < sd.ntiles; b += kSortThreads) {
    const uint32_t i = b + threadIdx.x;
    const uint64_t ti = 2 * (uint64_t)(sd.tile0 + i);
    const uint32_t e = i < sd.ntiles ? tcnt[ti] : 0;
    const uint32_t f = i < sd.ntiles ? tcnt[ti + 1] : 0;
    uint32_t te, tf;
    const uint32_t pe = block_excl_scan(e, sw, &te) + carry_e;
    const uint32_t pf = block_excl_scan(f, sw, &tf) + carry_f;
    if (i < sd.ntiles) {
      tcnt[ti] = pe;
      tcnt[ti + 1] = pf;
    }
    carry_e += te;
    carry_f += tf;
  }
  if (threadIdx.x == 0) {
    segtot[2 * s] = carry_e;
    segtot[2 * s + 1] = carry_f;
  }
}

// Entry and feature numbering.  Temporaries of segment s live at
// [sd.base + s, sd.base + s + G + 1).
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads)
k_rle_emit(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
           const KeyT* __restrict__ keys, const uint32_t* __restrict__ vals,
           const uint32_t* __restrict__ win2seq, const uint32_t* __restrict__ tcnt,
           uint32_t* __restrict__ estart, uint32_t* __restrict__ etseq,
           uint32_t* __restrict__ efid, uint32_t* __restrict__ fstart,
           uint32_t* __restrict__ ewin) {
  __shared__ uint32_t swe[kWarps], swf[kWarps];
  const uint32_t t = blockIdx.x;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t lt = t - sd.tile0;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt_mask = lanemask_lt();
  // Pass 1: per-warp totals.
  uint32_t we = 0, wf = 0;
#pragma unroll 4
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    bool ne = false, nf = false;
    uint32_t seq;
    if (idx < cnt) rle_flags<KeyT>(sd, (uint32_t)(beg + idx), keys, vals, win2seq, seq, ne, nf);
    we += __popc(__ballot_sync(0xffffffffu, ne));
    wf += __popc(__ballot_sync(0xffffffffu, nf));
  }
  if (lane == 0) {
    swe[w] = we;
    swf[w] = wf;
  }
  __syncthreads();
  uint32_t re = tcnt[2 * (uint64_t)t], rf = tcnt[2 * (uint64_t)t + 1];
  for (int i = 0; i < w; ++i) {
    re += swe[i];
    rf += swf[i];
  }
  const uint64_t tb = sd.base + s;
  // Pass 2: numbering and writes.  re / rf count entries / features that
  // start before the current element.
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    bool ne = false, nf = false;
    uint32_t seq = 0;
    if (idx < cnt) rle_flags<KeyT>(sd, (uint32_t)(beg + idx), keys, vals, win2seq, seq, ne, nf);
    const uint32_t be = __ballot_sync(0xffffffffu, ne);
    const uint32_t bf = __ballot_sync(0xffffffffu, nf);
    if (idx < cnt) {
      const uint32_t i = (uint32_t)(beg + idx);
      // Index of this element's entry / feature.
      const uint32_t e = re + __popc(be & lt_mask) - (ne ? 0u : 1u);
      const uint32_t f = rf + __popc(bf & lt_mask) - (nf ? 0u : 1u);
      ewin[sd.pool + vals[sd.base + i]] = ne ? e : kNone;
      if (ne) {
        estart[tb + e] = i;
        etseq[tb + e] = seq;
        efid[tb + e] = f;
      }
      if (nf) fstart[tb + f] = e;
      if (i + 1 == sd.G) {
        estart[tb + e + 1] = sd.G;
        fstart[tb + f + 1] = e + 1;
      }
    }
    re += __popc(be);
    rf += __popc(bf);
  }
}

// Pack entries: eseq = (sequence << 16) | count, efe = end of the entry's
// feature (exclusive entry index).
__global__ void __launch_bounds__(kSortThreads)
k_rle_final(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
            const uint32_t* __restrict__ segtot, const uint32_t* __restrict__ estart,
            const uint32_t* __restrict__ etseq, const uint32_t* __restrict__ efid,
            const uint32_t* __restrict__ fstart, uint32_t* __restrict__ eseq,
            uint32_t* __restrict__ efe) {
  const uint32_t t = blockIdx.x;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t lt = t - sd.tile0;
  const uint32_t E = segtot[2 * s];
  const uint64_t tb = sd.base + s;
  const uint64_t beg = (uint64_t)lt * kTile;
  for (uint32_t q = threadIdx.x; q < kTile; q += blockDim.x) {
    const uint64_t e = beg + q;
    if (e >= E) break;
    const uint32_t c = estart[tb + e + 1] - estart[tb + e];
    eseq[sd.pool + e] = (etseq[tb + e] << 16) | c;
    efe[sd.pool + e] = fstart[tb + efid[tb + e] + 1];
  }
}

template <typename KeyT>
void sort_pass_t(bool first, const SegDesc* segs, uint32_t nsegs,
                 const uint32_t* tile_seg, uint32_t ntiles,
                 const MaskDesc* masks, const uint64_t* fullkey,
                 const void* kin, const uint32_t* vin, void* kout,
                 uint32_t* vout, uint32_t* hist, int shift, int rbits,
                 cudaStream_t st) {
  const size_t radix = (size_t)1 << rbits;
  const size_t up_smem = radix * 4;
  const size_t dn_smem = (kWarps + 1) * radix * 4;
  const KeyT* ki = (const KeyT*)kin;
  KeyT* ko = (KeyT*)kout;
  if (first) {
    auto ku = k_upsweep<KeyT, true>;
    auto kd = k_downsweep<KeyT, true>;
    ku<<<ntiles, kSortThreads, up_smem, st>>>(segs, tile_seg, masks, fullkey, ki, hist, shift, rbits);
    k_seg_scan<<<nsegs, kSortThreads, 0, st>>>(segs, hist, rbits);
    kd<<<ntiles, kSortThreads, dn_smem, st>>>(segs, tile_seg, masks, fullkey, ki, vin, ko, vout, hist, shift, rbits);
  } else {
    auto ku = k_upsweep<KeyT, false>;
    auto kd = k_downsweep<KeyT, false>;
    ku<<<ntiles, kSortThreads, up_smem, st>>>(segs, tile_seg, masks, fullkey, ki, hist, shift, rbits);
    k_seg_scan<<<nsegs, kSortThreads, 0, st>>>(segs, hist, rbits);
    kd<<<ntiles, kSortThreads, dn_smem, st>>>(segs, tile_seg, masks, fullkey, ki, vin, ko, vout, hist, shift, rbits);
  }
}

template <typename KeyT>
void rle_t(const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg,
           uint32_t ntiles, const void* keys, const uint32_t* vals,
           const uint32_t* win2seq, uint32_t* tcnt, uint32_t* segtot,
           uint32_t* estart, uint32_t* etseq, uint32_t* efid,
           uint32_t* fstart, uint32_t* ewin, uint32_t* eseq, uint32_t* efe,
           cudaStream_t st) {
  const KeyT* k = (const KeyT*)keys;
  k_rle_count<KeyT><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, k, vals, win2seq, tcnt);
  k_rle_scan<<<nsegs, kSortThreads, 0, st>>>(segs, tcnt, segtot);
  k_rle_emit<KeyT><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, k, vals, win2seq, tcnt,
                                                    estart, etseq, efid, fstart, ewin);
  k_rle_final<<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, segtot, estart, etseq, efid,
                                               fstart, eseq, efe);
}

}  // namespace

int prep_init() {
  // Largest downsweep footprint: (warps + 1) x 2^kMaxRadixBits counters.
  const int smem = (kWarps + 1) * (1 << kMaxRadixBits) * 4;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return (int)e;
}

void launch_pack(const DsPack* d_ds, uint32_t nds, uint32_t nseq_total, int g,
                 int bits, int sigma, uint64_t* fullkey, uint32_t* win2seq,
                 uint32_t* status, cudaStream_t st) {
  if (nseq_total == 0) return;
  k_pack<<<nseq_total, 128, 0, st>>>(d_ds, nds, g, bits, sigma, fullkey, win2seq, status);
}

void launch_sort_pass(bool wide, bool first, const SegDesc* segs,
                      uint32_t nsegs, const uint32_t* tile_seg,
                      uint32_t ntiles, const MaskDesc* masks,
                      const uint64_t* fullkey, const void* kin,
                      const uint32_t* vin, void* kout, uint32_t* vout,
                      uint32_t* hist, int shift, int rbits, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    sort_pass_t<uint64_t>(first, segs, nsegs, tile_seg, ntiles, masks, fullkey, kin, vin, kout,
                          vout, hist, shift, rbits, st);
  else
    sort_pass_t<uint32_t>(first, segs, nsegs, tile_seg, ntiles, masks, fullkey, kin, vin, kout,
                          vout, hist, shift, rbits, st);
}

void launch_rle(bool wide, const SegDesc* segs, uint32_t nsegs,
                const uint32_t* tile_seg, uint32_t ntiles, const void* keys,
                const uint32_t* vals, const uint32_t* win2seq, uint32_t* tcnt,
                uint32_t* segtot, uint32_t* estart, uint32_t* etseq,
                uint32_t* efid, uint32_t* fstart, uint32_t* ewin,
                uint32_t* eseq, uint32_t* efe, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    rle_t<uint64_t>(segs, nsegs, tile_seg, ntiles, keys, vals, win2seq, tcnt, segtot, estart,
                    etseq, efid, fstart, ewin, eseq, efe, st);
  else
    rle_t<uint32_t>(segs, nsegs, tile_seg, ntiles, keys, vals, win2seq, tcnt, segtot, estart,
                    etseq, efid, fstart, ewin, eseq, efe, st);
}

}  // namespace gk
