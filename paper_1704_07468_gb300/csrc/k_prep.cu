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
// symbol in the most significant bits, b bits per symbol) and its window id
// (sequence << 16 | position of the window in the sequence; both fit 16
// bits, which the host checks).  Symbols >= sigma raise kErrBadCode.
__global__ void __launch_bounds__(128)
k_pack(const DsPack* __restrict__ ds, uint32_t nds, int g, int bits,
       int sigma, uint64_t* __restrict__ fullkey,
       uint32_t* __restrict__ wid, uint32_t* __restrict__ status) {
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
    wid[base + i] = (x << 16) | i;
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

// Masked key with the mask's runs held in registers (up to kRegRuns runs,
// i.e. M <= kRegRuns - 1 deleted positions; longer masks take the loop).
constexpr int kRegRuns = 6;

struct MaskRegs {
  uint32_t sh[kRegRuns];  // sr - sl: a run moves from bit sr of the full key to bit sl <= sr
  uint64_t mk[kRegRuns];  // the run's mask at its place in the masked key (msk << sl)
  bool fits;              // runs mode with at most kRegRuns runs
  bool fits32;            // ... every run within the full key's low 32 bits
};

__device__ __forceinline__ void mask_regs(const MaskDesc& md, MaskRegs& r) {
  r.fits = md.fold == 0 && md.nruns <= (uint32_t)kRegRuns;
  r.fits32 = r.fits;
#pragma unroll
  for (int i = 0; i < kRegRuns; ++i) {
    const bool on = (uint32_t)i < md.nruns;
    r.sh[i] = on ? md.sr[i] - md.sl[i] : 0u;
    r.mk[i] = on ? md.msk[i] << md.sl[i] : 0ull;
    if (on && md.sr[i] + (uint32_t)(64 - __clzll(md.msk[i])) > 32u) r.fits32 = false;
  }
}

// (full >> sr) & msk) << sl == (full >> (sr - sl)) & (msk << sl): one
// shift and one AND-OR per run, in 32-bit arithmetic when every run lies in
// the low 32 bits (the masked key then fits 32 bits as well).
__device__ __forceinline__ uint64_t masked_key_r(uint64_t full, const MaskRegs& r,
                                                 const MaskDesc& md) {
  if (!r.fits) return masked_key(full, md);
  if (r.fits32) {
    const uint32_t f = (uint32_t)full;
    uint32_t k = 0;
#pragma unroll
    for (int i = 0; i < kRegRuns; ++i) k |= (f >> r.sh[i]) & (uint32_t)r.mk[i];
    return k;
  }
  uint64_t k = 0;
#pragma unroll
  for (int i = 0; i < kRegRuns; ++i) k |= (full >> r.sh[i]) & r.mk[i];
  return k;
}

// Per-tile digit counts: hist[seg.hist + digit * ntiles + tile].  The first
// pass also cuts the masked keys out of the full g-mer keys and stores them
// in `kx`, which that pass's scatter then reads.
template <typename KeyT, bool kFirst>
__global__ void __launch_bounds__(kSortThreads)
k_upsweep(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
          const MaskDesc* __restrict__ masks, const uint64_t* __restrict__ fullkey,
          KeyT* __restrict__ kx, uint32_t* __restrict__ hist, int shift, int rbits) {
  extern __shared__ uint32_t sh[];
  __shared__ MaskDesc md;
  const uint32_t t = blockIdx.x;
  const SegDesc sd = segs[tile_seg[t]];
  const uint32_t lt = t - sd.tile0;
  const uint32_t radix = 1u << rbits;
  if (kFirst && threadIdx.x == 0) md = masks[sd.mask];
  for (uint32_t i = threadIdx.x; i < radix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  MaskRegs mr;
  if (kFirst) mask_regs(md, mr);
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    KeyT key;
    if (kFirst) {
      key = (KeyT)masked_key_r(fullkey[sd.win0 + beg + i], mr, md);
      kx[sd.base + beg + i] = key;
    } else {
      key = kx[sd.base + beg + i];
    }
    atomicAdd(&sh[(uint32_t)(key >> shift) & (radix - 1)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < radix; i += blockDim.x)
    hist[sd.hist + (uint64_t)i * sd.ntiles + lt] = sh[i];
}

// Grid (segments, digits / kWarps), one warp per (segment, digit):
// exclusive scan of the digit's per-tile counts of the segment (contiguous
// in the digit-major layout), in place; the digit's total to
// dtot[segment * radix + digit].  (A block per digit spent most of its time
// being scheduled: a segment has a few hundred tiles.)
__global__ void __launch_bounds__(kSortThreads)
k_digit_scan(const SegDesc* __restrict__ segs, uint32_t* __restrict__ hist, uint32_t* __restrict__ dtot,
             int rbits) {
  const uint32_t s = blockIdx.x;
  const uint32_t d = blockIdx.y * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (d >= (1u << rbits)) return;  // (the whole warp)
  const SegDesc sd = segs[s];
  uint32_t* __restrict__ h = hist + sd.hist + (uint64_t)d * sd.ntiles;
  uint32_t carry = 0;
  for (uint32_t b = 0; b < sd.ntiles; b += 32) {
    const uint32_t i = b + lane;
    const uint32_t v = i < sd.ntiles ? h[i] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (i < sd.ntiles) h[i] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) dtot[((uint64_t)s << rbits) + d] = carry;
}

// The same with a block per (segment, digit), four counts per thread: for
// segments of many tiles (grid (segments, digits)).
__global__ void __launch_bounds__(kSortThreads)
k_digit_scan_block(const SegDesc* __restrict__ segs, uint32_t* __restrict__ hist, uint32_t* __restrict__ dtot,
             int rbits) {
  __shared__ uint32_t sw[kWarps + 1];
  const uint32_t s = blockIdx.x, d = blockIdx.y;
  const SegDesc sd = segs[s];
  uint32_t* __restrict__ h = hist + sd.hist + (uint64_t)d * sd.ntiles;
  uint32_t carry = 0;
  for (uint32_t b = 0; b < sd.ntiles; b += kSortThreads * 4) {
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = b + threadIdx.x * 4 + q;
      v[q] = i < sd.ntiles ? h[i] : 0u;
      sum += v[q];
    }
    uint32_t tot;
    uint32_t pre = block_excl_scan(sum, sw, &tot) + carry;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = b + threadIdx.x * 4 + q;
      if (i < sd.ntiles) h[i] = pre;
      pre += v[q];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) dtot[((uint64_t)s << rbits) + d] = carry;
}

// One block per segment: the digit totals become the digits' starts
// (exclusive scan, in place).
__global__ void __launch_bounds__(kSortThreads)
k_digit_base(uint32_t* __restrict__ dtot, int rbits) {
  __shared__ uint32_t sw[kWarps + 1];
  const uint32_t radix = 1u << rbits;
  uint32_t* __restrict__ t = dtot + ((uint64_t)blockIdx.x << rbits);
  uint32_t carry = 0;
  for (uint32_t b = 0; b < radix; b += kSortThreads) {
    const uint32_t i = b + threadIdx.x;
    const uint32_t v = i < radix ? t[i] : 0u;
    uint32_t tot;
    const uint32_t pre = block_excl_scan(v, sw, &tot) + carry;
    if (i < radix) t[i] = pre;
    carry += tot;
  }
}

// Lanes of the warp holding the same digit as this lane: a warp multisplit
// by bit-sliced ballots (Ashkiani et al., "GPU Multisplit", PPoPP 2016), one
// ballot per digit bit plus one for validity, so that invalid lanes never
// join a valid lane's group.  kBits may exceed the digit width (the extra
// bits are zero in every lane).  On sm_103a this runs on the integer pipe;
// match.any, its one-instruction alternative, runs on the much narrower ADU
// pipe (see rank_items for how the two are mixed).
template <int kBits>
__device__ __forceinline__ uint32_t digit_peers(uint32_t dg, bool valid) {
  const uint32_t vb = __ballot_sync(0xffffffffu, valid);
  uint32_t peers = valid ? vb : ~vb;
#pragma unroll
  for (int b = 0; b < kBits; ++b) {
    const bool bit = (dg >> b) & 1u;
    const uint32_t v = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? v : ~v;
  }
  return peers;
}

// Rank of each item of a warp among the warp's items with the same digit,
// in element order: the group's leader reserves slots of the warp's running
// count for the digit with an atomic add, and the shuffle of its result is
// the convergence point that orders consecutive items.
template <int kBits, typename KeyT>
__device__ __forceinline__ void rank_items(const KeyT (&keys)[kSortIpt], uint32_t (&rk)[kSortIpt],
                                           uint32_t cnt, int w, int lane, int shift,
                                           uint32_t radix, uint32_t* wc) {
  const uint32_t lt_mask = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    const bool valid = idx < cnt;
    const uint32_t dg = valid ? ((uint32_t)(keys[j] >> shift) & (radix - 1)) : 0u;
    // Every fourth item takes match.any (ADU pipe), the others the ballots
    // (integer pipe), so that both pipes share the ranking work (measured
    // sort time against ballots alone: DNA large-M 5.35 -> 5.20 ms, protein
    // 4.54 -> 4.41, text 26.0 -> 25.0; match.any alone was ADU-bound, and
    // three items in four on it were slower than none).
    constexpr uint32_t kMatchItems = 0x1111u;
    const uint32_t peers = ((kMatchItems >> j) & 1u) ? __match_any_sync(0xffffffffu, valid ? dg : radix)
                                                     : digit_peers<kBits>(dg, valid);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&wc[w * radix + dg], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    rk[j] = base + __popc(peers & lt_mask);
  }
}

// Shared-memory footprint of the scatter kernel for a digit width.
__host__ __device__ constexpr size_t downsweep_smem(int rbits, int key_bytes) {
  return ((size_t)(kWarps + 2) << rbits) * 4 + (size_t)kTile * (key_bytes + 4);
}

// Stable scatter of one tile.  Warp w owns elements [w*32*IPT, (w+1)*32*IPT)
// and visits them as j*32 + lane, so the visiting order is the element
// order, and ranked within the warp by `rank_items`.  The tile is then laid out in digit
// order in shared memory and written out with consecutive threads on
// consecutive addresses of each digit's run.
// Resident blocks per SM: four for 32-bit keys, three for 64-bit keys
// (more would spill their register-held tiles).
template <typename KeyT, bool kFirst>
__global__ void __launch_bounds__(kSortThreads, sizeof(KeyT) == 8 ? 3 : 4)
k_downsweep(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
            const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin,
            KeyT* __restrict__ kout, uint32_t* __restrict__ vout,
            const uint32_t* __restrict__ hist, const uint32_t* __restrict__ dbase, int shift, int rbits) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t sw[kWarps + 1];
  const uint32_t radix = 1u << rbits;
  uint32_t* wc = sh;                     // kWarps x radix running counts
  uint32_t* gb = sh + kWarps * radix;    // global base of each digit in this tile, then
                                         // that base minus the digit's tile-local start
  uint32_t* ts = gb + radix;             // tile-local start of each digit
  KeyT* skey = (KeyT*)(ts + radix);      // tile in digit order
  uint32_t* sval = (uint32_t*)(skey + kTile);
  const uint32_t t = blockIdx.x;
  const uint32_t sx = tile_seg[t];
  const SegDesc sd = segs[sx];
  const uint32_t lt = t - sd.tile0;
  for (uint32_t i = threadIdx.x; i < kWarps * radix; i += blockDim.x) wc[i] = 0;
  for (uint32_t i = threadIdx.x; i < radix; i += blockDim.x)
    gb[i] = hist[sd.hist + (uint64_t)i * sd.ntiles + lt] + dbase[((uint64_t)sx << rbits) + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  const KeyT* __restrict__ ki = kin + sd.base + beg;
  const uint32_t* __restrict__ vi = vin + (kFirst ? sd.win0 : sd.base) + beg;
  KeyT keys[kSortIpt];
  uint32_t vals[kSortIpt];
  uint32_t rk[kSortIpt];
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    keys[j] = idx < cnt ? ki[idx] : (KeyT)0;
    vals[j] = idx < cnt ? vi[idx] : 0u;
  }
  // Ballots for 7, 8 or all digit bits (the digit width is uniform per launch).
  if (rbits <= 7)
    rank_items<7>(keys, rk, cnt, w, lane, shift, radix, wc);
  else if (rbits == 8)
    rank_items<8>(keys, rk, cnt, w, lane, shift, radix, wc);
  else
    rank_items<kMaxRadixBits>(keys, rk, cnt, w, lane, shift, radix, wc);
  __syncthreads();
  // Per digit: exclusive prefix over warps, and the digit's tile total.
  const uint32_t per = (radix + kSortThreads - 1) / kSortThreads;
  const uint32_t d0 = threadIdx.x * per;
  uint32_t mysum = 0;
  for (uint32_t q = 0; q < per; ++q) {
    const uint32_t dg = d0 + q;
    if (dg >= radix) break;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t c = wc[ww * radix + dg];
      wc[ww * radix + dg] = run;
      run += c;
    }
    ts[dg] = run;
    mysum += run;
  }
  // Tile-local digit starts: exclusive scan of the totals, folded into
  // every warp's offsets and into the global bases.
  uint32_t pre = block_excl_scan(mysum, sw, nullptr);
  for (uint32_t q = 0; q < per; ++q) {
    const uint32_t dg = d0 + q;
    if (dg >= radix) break;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) wc[ww * radix + dg] += pre;
    gb[dg] -= pre;
    pre += ts[dg];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    if (idx < cnt) {
      const uint32_t dg = (uint32_t)(keys[j] >> shift) & (radix - 1);
      const uint32_t lpos = wc[w * radix + dg] + rk[j];
      skey[lpos] = keys[j];
      sval[lpos] = vals[j];
    }
  }
  __syncthreads();
  KeyT* __restrict__ ko = kout + sd.base;
  uint32_t* __restrict__ vo = vout + sd.base;
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const KeyT k = skey[i];
    const uint32_t pos = gb[(uint32_t)(k >> shift) & (radix - 1)] + i;
    ko[pos] = k;
    vo[pos] = sval[i];
  }
}

// -------------------------------------------------------------- onesweep --
//
// The same stable LSD sort with one read of the keys per pass (Adinets and
// Merrill, "Onesweep: a faster least significant digit radix sort for GPUs",
// 2022): k_os_hist cuts the masked keys out of the full g-mer keys and
// counts the digits of every pass of every segment at once; k_os_base turns
// the counts into each digit's start in its segment; then one k_os_scatter
// launch per pass ranks each tile exactly as k_downsweep does and finds its
// digits' offsets among the segment's earlier tiles by a decoupled
// look-back: every tile publishes, per digit, first its own count
// (aggregate) and then its inclusive prefix, and a tile sums its
// predecessors' published values, newest first, until it meets a prefix.
// Tiles are taken in order from a counter, so a tile only ever waits on
// tiles that running or finished blocks have taken.  Waits are bounded: a
// wait that runs out raises kErrTimeout (the result is then invalid and the
// call fails) and the tile goes on.
//
// A status word holds (epoch << 48) | (kind << 46) | value: the epoch
// numbers the pass within the call (the words are cleared once per call),
// the kind is 1 for an aggregate and 2 for an inclusive prefix.

constexpr uint64_t kOsAgg = 1ull << 46, kOsIncl = 2ull << 46;
constexpr uint64_t kOsValue = (1ull << 46) - 1;
constexpr long long kOsWaitCycles = 4000000000ll;  // about 2 s
// Predecessor words loaded together in the look-back.  One at a time
// measured fastest (4, 8 and 16 raise register pressure and spill).
constexpr int kOsBatch = 1;

__device__ __forceinline__ void os_store(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t os_load(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads)
k_os_hist(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
          const MaskDesc* __restrict__ masks, const uint64_t* __restrict__ fullkey,
          KeyT* __restrict__ kx, uint32_t* __restrict__ dcount, OsPasses ps) {
  __shared__ uint32_t sh[kOsMaxPasses * kOsRadix];
  __shared__ MaskDesc md;
  __shared__ uint32_t s_shift[kOsMaxPasses], s_mask[kOsMaxPasses];
  const uint32_t t = blockIdx.x;
  const uint32_t sx = tile_seg[t];
  const SegDesc sd = segs[sx];
  const uint32_t lt = t - sd.tile0;
  if (threadIdx.x == 0) md = masks[sd.mask];
  if (threadIdx.x < (uint32_t)ps.np) {
    s_shift[threadIdx.x] = (uint32_t)ps.shift[threadIdx.x];
    s_mask[threadIdx.x] = (1u << ps.bits[threadIdx.x]) - 1u;
  }
  for (uint32_t i = threadIdx.x; i < (uint32_t)ps.np * kOsRadix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  MaskRegs mr;
  mask_regs(md, mr);
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const KeyT key = (KeyT)masked_key_r(fullkey[sd.win0 + beg + i], mr, md);
    kx[sd.base + beg + i] = key;
    for (int q = 0; q < ps.np; ++q) atomicAdd(&sh[q * kOsRadix + ((uint32_t)(key >> s_shift[q]) & s_mask[q])], 1u);
  }
  __syncthreads();
  uint32_t* __restrict__ dc = dcount + (uint64_t)sx * ps.np * kOsRadix;
  for (uint32_t i = threadIdx.x; i < (uint32_t)ps.np * kOsRadix; i += blockDim.x)
    if (sh[i]) atomicAdd(&dc[i], sh[i]);
}

// Grid (segments, passes): each digit's start in its segment, in place.
__global__ void __launch_bounds__(kSortThreads)
k_os_base(uint32_t* __restrict__ dcount, int np) {
  __shared__ uint32_t sw[kWarps + 1];
  uint32_t* __restrict__ d = dcount + ((uint64_t)blockIdx.x * np + blockIdx.y) * kOsRadix;
  static_assert(kOsRadix == kSortThreads, "one digit per thread");
  const uint32_t v = d[threadIdx.x];
  d[threadIdx.x] = block_excl_scan(v, sw, nullptr);
}

template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads, sizeof(KeyT) == 8 ? 3 : 4)
k_os_scatter(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
             const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin, bool first,
             KeyT* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* __restrict__ dbase,
             int np, int q, int shift, int rbits, uint64_t* __restrict__ st, uint32_t* __restrict__ ctr,
             uint32_t epoch, uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t sw[kWarps + 1];
  __shared__ uint32_t s_tile;
  const uint32_t radix = 1u << rbits;
  uint32_t* wc = sh;                     // kWarps x radix running counts
  uint32_t* gb = sh + kWarps * radix;    // global position of each digit's first element, minus
                                         // its tile-local start
  uint32_t* ts = gb + radix;             // the tile's count of each digit
  KeyT* skey = (KeyT*)(ts + radix);      // tile in digit order
  uint32_t* sval = (uint32_t*)(skey + kTile);
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
  for (uint32_t i = threadIdx.x; i < kWarps * radix; i += blockDim.x) wc[i] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t sx = tile_seg[t];
  const SegDesc sd = segs[sx];
  const uint32_t lt = t - sd.tile0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  const KeyT* __restrict__ ki = kin + sd.base + beg;
  const uint32_t* __restrict__ vi = vin + (first ? sd.win0 : sd.base) + beg;
  KeyT keys[kSortIpt];
  uint32_t vals[kSortIpt];
  uint32_t rk[kSortIpt];
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    keys[j] = idx < cnt ? ki[idx] : (KeyT)0;
    vals[j] = idx < cnt ? vi[idx] : 0u;
  }
  if (rbits <= 7)
    rank_items<7>(keys, rk, cnt, w, lane, shift, radix, wc);
  else
    rank_items<8>(keys, rk, cnt, w, lane, shift, radix, wc);
  __syncthreads();
  // Per digit (one per thread): exclusive prefix over warps and the tile's
  // count; publish the count, then look back for the earlier tiles' sum.
  const uint32_t dg = threadIdx.x;
  uint32_t run = 0;
  if (dg < radix) {
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t c = wc[ww * radix + dg];
      wc[ww * radix + dg] = run;
      run += c;
    }
    ts[dg] = run;
  }
  const uint64_t E = (uint64_t)epoch << 48;
  uint64_t* __restrict__ my = st + (uint64_t)t * kOsRadix;
  uint32_t excl = 0;
  if (dg < radix) {
    if (lt == 0) {
      os_store(&my[dg], E | kOsIncl | run);
    } else {
      os_store(&my[dg], E | kOsAgg | run);
      // Predecessors in batches of kOsBatch: their words are loaded
      // together, then taken newest first; a word not yet published is
      // polled until it is (the segment's first tile publishes a prefix at
      // once, so the walk ends there at the latest).
      uint32_t j = t;  // next predecessor is j - 1
      bool done = false;
      while (!done) {
        const uint32_t nb = min((uint32_t)kOsBatch, j - sd.tile0);
        uint64_t v[kOsBatch];
#pragma unroll
        for (int i = 0; i < kOsBatch; ++i)
          v[i] = (uint32_t)i < nb ? os_load(&st[(uint64_t)(j - 1 - i) * kOsRadix + dg]) : 0ull;
#pragma unroll
        for (int i = 0; i < kOsBatch; ++i) {
          if (done || (uint32_t)i >= nb) continue;
          const long long t0 = clock64();
          while (!((v[i] >> 48) == epoch && (v[i] & (kOsAgg | kOsIncl)))) {
            if (clock64() - t0 > kOsWaitCycles) {
              atomicOr(status, kErrTimeout);
              v[i] = ((uint64_t)epoch << 48) | kOsIncl;  // give up: treat as a zero prefix
              break;
            }
            v[i] = os_load(&st[(uint64_t)(j - 1 - i) * kOsRadix + dg]);
          }
          excl += (uint32_t)(v[i] & kOsValue);
          if (v[i] & kOsIncl) done = true;
        }
        j -= nb;
        if (j == sd.tile0) done = true;
      }
      os_store(&my[dg], E | kOsIncl | (uint64_t)(excl + run));
    }
  }
  // Tile-local digit starts: exclusive scan of the counts, folded into the
  // warps' offsets and the global positions.
  const uint32_t pre = block_excl_scan(dg < radix ? run : 0u, sw, nullptr);
  if (dg < radix) {
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) wc[ww * radix + dg] += pre;
    gb[dg] = dbase[((uint64_t)sx * np + q) * kOsRadix + dg] + excl - pre;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    if (idx < cnt) {
      const uint32_t d = (uint32_t)(keys[j] >> shift) & (radix - 1);
      const uint32_t lpos = wc[w * radix + d] + rk[j];
      skey[lpos] = keys[j];
      sval[lpos] = vals[j];
    }
  }
  __syncthreads();
  KeyT* __restrict__ ko = kout + sd.base;
  uint32_t* __restrict__ vo = vout + sd.base;
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const KeyT k = skey[i];
    const uint32_t pos = gb[(uint32_t)(k >> shift) & (radix - 1)] + i;
    if (pos < sd.G) {  // (only a look-back that ran out can miss the segment)
      ko[pos] = k;
      vo[pos] = sval[i];
    } else {
      atomicOr(status, kErrBadEntry);
    }
  }
}

// ------------------------------------------------------------ run-length --

// Loads the elements a warp owns in a tile (element w*32*IPT + j*32 + lane)
// with their sequence ids, and flags: a new entry starts where the (key,
// sequence) pair changes, a new feature where the key changes.  The
// predecessor comes from the neighbouring lane by shuffle; only the warp's
// first element reads its predecessor from memory.
template <typename KeyT, int kIpt = kSortIpt>
__device__ __forceinline__ void rle_load_flags(const SegDesc& sd, uint64_t beg, uint32_t cnt,
                                               int w, int lane,
                                               const KeyT* __restrict__ keys,
                                               const uint32_t* __restrict__ vals,
                                               uint32_t (&vv)[kIpt], uint32_t& ne_bits,
                                               uint32_t& nf_bits) {
  // Predecessor of the warp's first element.
  const uint64_t first = beg + (uint64_t)w * 32 * kIpt;
  KeyT k_prev = 0;
  uint32_t s_prev = kNone;
  if (lane == 0 && first > 0 && first - beg < cnt) {
    k_prev = keys[sd.base + first - 1];
    s_prev = vals[sd.base + first - 1] >> 16;
  }
  ne_bits = nf_bits = 0;
#pragma unroll
  for (int j = 0; j < kIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kIpt + j * 32 + lane;
    KeyT kj = 0;
    vv[j] = 0;
    if (idx < cnt) {
      kj = keys[sd.base + beg + idx];
      vv[j] = vals[sd.base + beg + idx];
    }
    const uint32_t sj = vv[j] >> 16;  // the sequence (only read where idx < cnt)
    KeyT kp = __shfl_up_sync(0xffffffffu, kj, 1);
    uint32_t sp = __shfl_up_sync(0xffffffffu, sj, 1);
    const KeyT k31 = __shfl_sync(0xffffffffu, kj, 31);
    const uint32_t s31 = __shfl_sync(0xffffffffu, sj, 31);
    if (lane == 0) {
      kp = k_prev;
      sp = s_prev;
    }
    if (idx < cnt) {
      const bool at0 = beg + idx == 0;
      const bool nf = at0 || kj != kp;
      const bool ne = nf || sj != sp;
      nf_bits |= (uint32_t)nf << j;
      ne_bits |= (uint32_t)ne << j;
    }
    k_prev = k31;  // lane 0 of the next item follows lane 31 of this one
    s_prev = s31;
  }
}

template <typename KeyT, int kIpt = kSortIpt>
__global__ void __launch_bounds__(kTile / kIpt)
k_rle_count(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
            const KeyT* __restrict__ keys, const uint32_t* __restrict__ vals,
            uint32_t* __restrict__ tcnt) {
  constexpr int kW = kTile / kIpt / 32;
  __shared__ uint32_t sw[2][kW];
  const uint32_t t = blockIdx.x;
  const SegDesc sd = segs[tile_seg[t]];
  const uint32_t lt = t - sd.tile0;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t vv[kIpt], ne_bits, nf_bits;
  rle_load_flags<KeyT, kIpt>(sd, beg, cnt, w, lane, keys, vals, vv, ne_bits, nf_bits);
  uint32_t ce = __popc(ne_bits), cf = __popc(nf_bits);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ce += __shfl_xor_sync(0xffffffffu, ce, o);
    cf += __shfl_xor_sync(0xffffffffu, cf, o);
  }
  if (lane == 0) {
    sw[0][w] = ce;
    sw[1][w] = cf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int i = 0; i < kW; ++i) {
      a += sw[0][i];
      b += sw[1][i];
    }
    tcnt[2 * (uint64_t)t] = a;
    tcnt[2 * (uint64_t)t + 1] = b;
  }
}

// Exclusive scan of the (entries, features) counts of each segment's tiles;
// totals go to segtot[2 * s] (E) and segtot[2 * s + 1] (F), and E is added
// to *ecount when it is given (the call's work figure).
__global__ void __launch_bounds__(kSortThreads)
k_rle_scan(const SegDesc* __restrict__ segs, uint32_t* __restrict__ tcnt,
           uint32_t* __restrict__ segtot, unsigned long long* __restrict__ ecount) {
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
    if (ecount) atomicAdd(ecount, (unsigned long long)carry_e);
  }
}

// Entry and feature numbering.  Temporaries of segment s live at
// [sd.base + s, sd.base + s + G + 1).
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads, 3)
k_rle_emit(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
           const KeyT* __restrict__ keys, const uint32_t* __restrict__ vals,
           const DsPack* __restrict__ dsp, const uint32_t* __restrict__ tcnt,
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
  const uint32_t* __restrict__ woff = dsp[sd.ds].woff;
  uint32_t vv[kSortIpt], ne_bits, nf_bits;
  rle_load_flags<KeyT>(sd, beg, cnt, w, lane, keys, vals, vv, ne_bits, nf_bits);
  uint32_t we = __popc(ne_bits), wf = __popc(nf_bits);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    we += __shfl_xor_sync(0xffffffffu, we, o);
    wf += __shfl_xor_sync(0xffffffffu, wf, o);
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
  // re / rf count entries / features that start before the current item.
#pragma unroll
  for (int j = 0; j < kSortIpt; ++j) {
    const uint32_t idx = (uint32_t)w * 32 * kSortIpt + j * 32 + lane;
    const bool ne = (ne_bits >> j) & 1u, nf = (nf_bits >> j) & 1u;
    const uint32_t be = __ballot_sync(0xffffffffu, ne);
    const uint32_t bf = __ballot_sync(0xffffffffu, nf);
    if (idx < cnt) {
      const uint32_t i = (uint32_t)(beg + idx);
      const uint32_t e = re + __popc(be & lt_mask) - (ne ? 0u : 1u);
      const uint32_t f = rf + __popc(bf & lt_mask) - (nf ? 0u : 1u);
      ewin[sd.pool + woff[vv[j] >> 16] + (vv[j] & 0xFFFFu)] = ne ? e : kNone;
      if (ne) {
        estart[tb + e] = i;
        etseq[tb + e] = vv[j] >> 16;
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

// Gram-engine variant of k_rle_emit + k_rle_final: writes ewin and the
// packed entries directly.  For an entry e starting at element i:
//   eseq[e] = (sequence << 16) | count, count = (next entry start) - i;
//   efe[e]  = first entry of the next feature.
// A feature held by one sequence only adds count^2 to that sequence's
// diagonal; when its count is known here, ewin of its first window holds
// kSingleTag | count instead of the entry (see k_accum).
// Both "next" starts are found by a backward pass over the tile's items
// (ballots within a warp, per-warp summaries across warps).  The last entry
// of a tile, and the entries of the tile's last feature, may end in a later
// tile: their count is left 0 / their efe unwritten, and the tile's record
// trec[t * kRecWords ..] = {first entry element, last entry element, its
// entry, first feature's entry, last feature's entry} (tile-local element
// indices, kNone where absent) lets k_rle_fix complete them.
template <typename KeyT, int kIpt = kSortIpt>
__global__ void __launch_bounds__(kTile / kIpt, kIpt == kSortIpt ? 5 : 4)
k_rle_emit_gram(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
                const KeyT* __restrict__ keys, const uint32_t* __restrict__ vals,
                const DsPack* __restrict__ dsp, const uint32_t* __restrict__ tcnt,
                uint32_t* __restrict__ trec, uint32_t* __restrict__ ewin,
                uint32_t* __restrict__ eseq, uint32_t* __restrict__ efe) {
  // Per warp: entries, first / last entry element (warp-local), and the
  // number of the warp's entries before its first / last feature start.
  constexpr int kW = kTile / kIpt / 32;
  __shared__ uint32_t swe[kW], sfe[kW], sle[kW], sff[kW], slf[kW];
  const uint32_t t = blockIdx.x;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t lt = t - sd.tile0;
  const uint64_t beg = (uint64_t)lt * kTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kTile, sd.G - beg);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t gt_mask = lane == 31 ? 0u : (0xFFFFFFFFu << (lane + 1));
  const uint32_t* __restrict__ woff = dsp[sd.ds].woff;
  uint32_t vv[kIpt], ne_bits, nf_bits;
  rle_load_flags<KeyT, kIpt>(sd, beg, cnt, w, lane, keys, vals, vv, ne_bits, nf_bits);
  {
    uint32_t nen = 0, fe = kNone, le = kNone, ff = kNone, lf = kNone;
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
      const uint32_t be = __ballot_sync(0xffffffffu, (ne_bits >> j) & 1u);
      const uint32_t bf = __ballot_sync(0xffffffffu, (nf_bits >> j) & 1u);
      if (be) {
        if (fe == kNone) fe = j * 32 + __ffs(be) - 1;
        le = j * 32 + 31 - __clz(be);
      }
      if (bf) {
        const uint32_t l0 = __ffs(bf) - 1, l1 = 31 - __clz(bf);
        if (ff == kNone) ff = nen + __popc(be & ((1u << l0) - 1u));
        lf = nen + __popc(be & ((1u << l1) - 1u));
      }
      nen += __popc(be);
    }
    if (lane == 0) {
      swe[w] = nen;
      sfe[w] = fe;
      sle[w] = le;
      sff[w] = ff;
      slf[w] = lf;
    }
  }
  __syncthreads();
  constexpr uint32_t kWarpElems = 32 * kIpt;
  const uint32_t e0 = tcnt[2 * (uint64_t)t];  // entries of the segment before this tile
  uint32_t re = e0;                           // entries before warp w
  for (int i = 0; i < w; ++i) re += swe[i];
  // First entry element (tile-local) and first feature start (entry index)
  // after warp w.
  uint32_t cne = kNone, cnf = kNone;
  {
    uint32_t r = re + swe[w];
    for (int i = w + 1; i < kW; ++i) {
      if (cne == kNone && sfe[i] != kNone) cne = i * kWarpElems + sfe[i];
      if (cnf == kNone && sff[i] != kNone) cnf = r + sff[i];
      r += swe[i];
    }
  }
  if (threadIdx.x == 0) {
    uint32_t r = e0, fe = kNone, le = kNone, le_e = kNone, ff = kNone, lf = kNone;
    for (int i = 0; i < kW; ++i) {
      if (sfe[i] != kNone) {
        if (fe == kNone) fe = i * kWarpElems + sfe[i];
        le = i * kWarpElems + sle[i];
        le_e = r + swe[i] - 1;
      }
      if (sff[i] != kNone) {
        if (ff == kNone) ff = r + sff[i];
        lf = r + slf[i];
      }
      r += swe[i];
    }
    uint32_t* rec = trec + (uint64_t)t * kRecWords;
    rec[0] = fe;
    rec[1] = le;
    rec[2] = le_e;
    rec[3] = ff;
    rec[4] = lf;
  }
  re += swe[w];  // entries before the item after the current one (walking back)
#pragma unroll
  for (int j = kIpt - 1; j >= 0; --j) {
    const bool ne = (ne_bits >> j) & 1u, nf = (nf_bits >> j) & 1u;
    const uint32_t be = __ballot_sync(0xffffffffu, ne);
    const uint32_t bf = __ballot_sync(0xffffffffu, nf);
    re -= __popc(be);  // entries before item j
    const uint32_t item0 = (uint32_t)w * kWarpElems + j * 32;
    const uint32_t idx = item0 + lane;
    if (idx < cnt) {
      const uint32_t e = re + __popc(be & lt_mask);
      uint32_t wv = kNone;
      if (ne) {
        const uint32_t hb = be & gt_mask;
        const uint32_t nxt = hb ? item0 + __ffs(hb) - 1 : cne;
        const uint32_t cv = nxt == kNone ? 0u : nxt - idx;
        eseq[sd.pool + e] = (vv[j] & 0xFFFF0000u) | cv;
        const uint32_t hf = bf & gt_mask;
        const uint32_t fend = hf ? re + __popc(be & ((1u << (__ffs(hf) - 1)) - 1u)) : cnf;
        if (fend != kNone) efe[sd.pool + e] = fend;
        wv = (nf && fend == e + 1 && cv != 0u) ? (kSingleTag | cv) : e;
      }
      ewin[sd.pool + woff[vv[j] >> 16] + (vv[j] & 0xFFFFu)] = wv;
    }
    if (be) cne = item0 + __ffs(be) - 1;
    if (bf) cnf = re + __popc(be & ((1u << (__ffs(bf) - 1)) - 1u));
  }
}

// Completes what k_rle_emit_gram left open at tile ends: one warp per
// tile.  The tile's last entry runs to the first entry element of a later
// tile of the segment (else to the segment's end); the entries of its last
// feature, up to the first feature start of a later tile (else the
// segment's entry count), get that start as their feature end.
__global__ void __launch_bounds__(256)
k_rle_fix(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg, uint32_t ntiles,
          const uint32_t* __restrict__ segtot, const uint32_t* __restrict__ trec,
          uint32_t* __restrict__ eseq, uint32_t* __restrict__ efe) {
  const uint32_t t = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t tend = sd.tile0 + sd.ntiles;
  const uint32_t* rec = trec + (uint64_t)t * kRecWords;
  const uint32_t le = rec[1], le_e = rec[2], lf = rec[4];
  if (le != kNone) {
    uint32_t end = sd.G;
    for (uint32_t u0 = t + 1; u0 < tend; u0 += 32) {
      const uint32_t u = u0 + lane;
      const uint32_t f = u < tend ? trec[(uint64_t)u * kRecWords] : kNone;
      const uint32_t b = __ballot_sync(0xffffffffu, f != kNone);
      if (b) {
        const uint32_t L = __ffs(b) - 1;
        end = (u0 + L - sd.tile0) * (uint32_t)kTile + __shfl_sync(0xffffffffu, f, L);
        break;
      }
    }
    if (lane == 0) eseq[sd.pool + le_e] += end - ((t - sd.tile0) * (uint32_t)kTile + le);
  }
  if (lf != kNone) {
    uint32_t fend = segtot[2 * (uint64_t)s];
    for (uint32_t u0 = t + 1; u0 < tend; u0 += 32) {
      const uint32_t u = u0 + lane;
      const uint32_t f = u < tend ? trec[(uint64_t)u * kRecWords + 3] : kNone;
      const uint32_t b = __ballot_sync(0xffffffffu, f != kNone);
      if (b) {
        fend = __shfl_sync(0xffffffffu, f, __ffs(b) - 1);
        break;
      }
    }
    for (uint32_t e = lf + lane; e < fend; e += 32) efe[sd.pool + e] = fend;
  }
}

template <typename KeyT>
void sort_pass_t(bool first, const SegDesc* segs, uint32_t nsegs,
                 const uint32_t* tile_seg, uint32_t ntiles,
                 const MaskDesc* masks, const uint64_t* fullkey,
                 void* kin, const uint32_t* vin, void* kout,
                 uint32_t* vout, uint32_t* hist, uint32_t* dtot, int shift, int rbits,
                 cudaStream_t st) {
  const size_t radix = (size_t)1 << rbits;
  // A warp per digit while segments average at most 256 tiles, else a block.
  const bool warp_scan = ntiles <= 256u * nsegs;
  const dim3 scan_grid(nsegs, (unsigned)(warp_scan ? (radix + kWarps - 1) / kWarps : radix));
  const size_t up_smem = radix * 4;
  const size_t dn_smem = downsweep_smem(rbits, (int)sizeof(KeyT));
  KeyT* ki = (KeyT*)kin;
  KeyT* ko = (KeyT*)kout;
  if (first) {
    k_upsweep<KeyT, true><<<ntiles, kSortThreads, up_smem, st>>>(segs, tile_seg, masks, fullkey, ki,
                                                                  hist, shift, rbits);
    if (warp_scan)
      k_digit_scan<<<scan_grid, kSortThreads, 0, st>>>(segs, hist, dtot, rbits);
    else
      k_digit_scan_block<<<scan_grid, kSortThreads, 0, st>>>(segs, hist, dtot, rbits);
    k_digit_base<<<nsegs, kSortThreads, 0, st>>>(dtot, rbits);
    k_downsweep<KeyT, true><<<ntiles, kSortThreads, dn_smem, st>>>(segs, tile_seg, ki, vin, ko, vout,
                                                                    hist, dtot, shift, rbits);
  } else {
    k_upsweep<KeyT, false><<<ntiles, kSortThreads, up_smem, st>>>(segs, tile_seg, masks, fullkey, ki,
                                                                   hist, shift, rbits);
    if (warp_scan)
      k_digit_scan<<<scan_grid, kSortThreads, 0, st>>>(segs, hist, dtot, rbits);
    else
      k_digit_scan_block<<<scan_grid, kSortThreads, 0, st>>>(segs, hist, dtot, rbits);
    k_digit_base<<<nsegs, kSortThreads, 0, st>>>(dtot, rbits);
    k_downsweep<KeyT, false><<<ntiles, kSortThreads, dn_smem, st>>>(segs, tile_seg, ki, vin, ko, vout,
                                                                     hist, dtot, shift, rbits);
  }
}

template <typename KeyT>
void rle_head_t(const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg,
                uint32_t ntiles, const void* keys, const uint32_t* vals,
                const DsPack* dsp, uint32_t* tcnt, uint32_t* segtot,
                uint32_t* estart, uint32_t* etseq, uint32_t* efid,
                uint32_t* fstart, uint32_t* ewin, cudaStream_t st) {
  const KeyT* k = (const KeyT*)keys;
  k_rle_count<KeyT><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, k, vals, tcnt);
  k_rle_scan<<<nsegs, kSortThreads, 0, st>>>(segs, tcnt, segtot, nullptr);
  k_rle_emit<KeyT><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, k, vals, dsp, tcnt,
                                                    estart, etseq, efid, fstart, ewin);
}

template <typename KeyT, int kIpt>
void rle_gram_t(const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg, uint32_t ntiles,
                const void* keys, const uint32_t* vals, const DsPack* dsp, uint32_t* tcnt,
                uint32_t* segtot, uint32_t* trec, uint32_t* ewin, uint32_t* eseq, uint32_t* efe,
                unsigned long long* ecount, cudaStream_t st) {
  const KeyT* k = (const KeyT*)keys;
  k_rle_count<KeyT, kIpt><<<ntiles, kTile / kIpt, 0, st>>>(segs, tile_seg, k, vals, tcnt);
  k_rle_scan<<<nsegs, kSortThreads, 0, st>>>(segs, tcnt, segtot, ecount);
  k_rle_emit_gram<KeyT, kIpt><<<ntiles, kTile / kIpt, 0, st>>>(segs, tile_seg, k, vals, dsp, tcnt, trec,
                                                               ewin, eseq, efe);
  k_rle_fix<<<(ntiles + 7) / 8, 256, 0, st>>>(segs, tile_seg, ntiles, segtot, trec, eseq, efe);
}

}  // namespace

int prep_init() {
  // Largest scatter footprint: the widest digit with 8-byte keys.
  const int big = (int)downsweep_smem(kMaxRadixBits, 8);
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  e = e ? e : cudaFuncSetAttribute(k_downsweep<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  const int os = (int)downsweep_smem(8, 8);
  e = e ? e : cudaFuncSetAttribute(k_os_scatter<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, os);
  e = e ? e : cudaFuncSetAttribute(k_os_scatter<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, os);
  return (int)e;
}

void launch_pack(const DsPack* d_ds, uint32_t nds, uint32_t nseq_total, int g,
                 int bits, int sigma, uint64_t* fullkey, uint32_t* wid,
                 uint32_t* status, cudaStream_t st) {
  if (nseq_total == 0) return;
  k_pack<<<nseq_total, 128, 0, st>>>(d_ds, nds, g, bits, sigma, fullkey, wid, status);
}

void launch_os_hist(bool wide, const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg,
                    uint32_t ntiles, const MaskDesc* masks, const uint64_t* fullkey, void* kx,
                    uint32_t* dcount, const OsPasses& ps, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    k_os_hist<uint64_t><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, masks, fullkey, (uint64_t*)kx, dcount, ps);
  else
    k_os_hist<uint32_t><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, masks, fullkey, (uint32_t*)kx, dcount, ps);
  k_os_base<<<dim3(nsegs, ps.np), kSortThreads, 0, st>>>(dcount, ps.np);
}

void launch_os_scatter(bool wide, bool first, const SegDesc* segs, const uint32_t* tile_seg,
                       uint32_t ntiles, const void* kin, const uint32_t* vin, void* kout,
                       uint32_t* vout, const uint32_t* dbase, int np, int q, int shift, int rbits,
                       uint64_t* st, uint32_t* ctr, uint32_t epoch, uint32_t* status, cudaStream_t stm) {
  if (ntiles == 0) return;
  const size_t smem = downsweep_smem(rbits, wide ? 8 : 4);
  if (wide)
    k_os_scatter<uint64_t><<<ntiles, kSortThreads, smem, stm>>>(segs, tile_seg, (const uint64_t*)kin, vin, first,
                                                                (uint64_t*)kout, vout, dbase, np, q, shift, rbits,
                                                                st, ctr, epoch, status);
  else
    k_os_scatter<uint32_t><<<ntiles, kSortThreads, smem, stm>>>(segs, tile_seg, (const uint32_t*)kin, vin, first,
                                                                (uint32_t*)kout, vout, dbase, np, q, shift, rbits,
                                                                st, ctr, epoch, status);
}

void launch_sort_pass(bool wide, bool first, const SegDesc* segs,
                      uint32_t nsegs, const uint32_t* tile_seg,
                      uint32_t ntiles, const MaskDesc* masks,
                      const uint64_t* fullkey, void* kin,
                      const uint32_t* vin, void* kout, uint32_t* vout,
                      uint32_t* hist, uint32_t* dtot, int shift, int rbits, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    sort_pass_t<uint64_t>(first, segs, nsegs, tile_seg, ntiles, masks, fullkey, kin, vin, kout,
                          vout, hist, dtot, shift, rbits, st);
  else
    sort_pass_t<uint32_t>(first, segs, nsegs, tile_seg, ntiles, masks, fullkey, kin, vin, kout,
                          vout, hist, dtot, shift, rbits, st);
}

void launch_rle_head(bool wide, const SegDesc* segs, uint32_t nsegs,
                     const uint32_t* tile_seg, uint32_t ntiles, const void* keys,
                     const uint32_t* vals, const DsPack* dsp, uint32_t* tcnt,
                     uint32_t* segtot, uint32_t* estart, uint32_t* etseq,
                     uint32_t* efid, uint32_t* fstart, uint32_t* ewin, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    rle_head_t<uint64_t>(segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, estart,
                         etseq, efid, fstart, ewin, st);
  else
    rle_head_t<uint32_t>(segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, estart,
                         etseq, efid, fstart, ewin, st);
}

void launch_rle_gram(bool wide, const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg,
                     uint32_t ntiles, const void* keys, const uint32_t* vals, const DsPack* dsp,
                     uint32_t* tcnt, uint32_t* segtot, uint32_t* trec, uint32_t* ewin,
                     uint32_t* eseq, uint32_t* efe, unsigned long long* ecount, int items,
                     cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide && items == 8)
    rle_gram_t<uint64_t, 8>(segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, trec, ewin,
                            eseq, efe, ecount, st);
  else if (wide)
    rle_gram_t<uint64_t, kSortIpt>(segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, trec, ewin,
                                   eseq, efe, ecount, st);
  else if (items == 8)
    rle_gram_t<uint32_t, 8>(segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, trec, ewin,
                            eseq, efe, ecount, st);
  else
    rle_gram_t<uint32_t, kSortIpt>(segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, trec, ewin,
                                   eseq, efe, ecount, st);
}

void launch_rle_final(const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                      const uint32_t* segtot, const uint32_t* estart,
                      const uint32_t* etseq, const uint32_t* efid,
                      const uint32_t* fstart, uint32_t* eseq, uint32_t* efe,
                      cudaStream_t st) {
  if (ntiles == 0) return;
  k_rle_final<<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, segtot, estart, etseq, efid,
                                               fstart, eseq, efe);
}

void launch_rle(bool wide, const SegDesc* segs, uint32_t nsegs,
                const uint32_t* tile_seg, uint32_t ntiles, const void* keys,
                const uint32_t* vals, const DsPack* dsp, uint32_t* tcnt,
                uint32_t* segtot, uint32_t* estart, uint32_t* etseq,
                uint32_t* efid, uint32_t* fstart, uint32_t* ewin,
                uint32_t* eseq, uint32_t* efe, cudaStream_t st) {
  launch_rle_head(wide, segs, nsegs, tile_seg, ntiles, keys, vals, dsp, tcnt, segtot, estart,
                  etseq, efid, fstart, ewin, st);
  launch_rle_final(segs, tile_seg, ntiles, segtot, estart, etseq, efid, fstart, eseq, efe, st);
}

}  // namespace gk
