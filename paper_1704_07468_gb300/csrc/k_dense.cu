// Dense levels: C_m += F^T F as a dense contraction on the tensor cores
// (tcgen05.mma, kind::f8f6f4 with e4m3 operands, f32 accumulators in
// tensor memory).
//
// For one mask the count matrix F has a row per feature and a column per
// sequence, and countAndUpdate adds F^T F to C_m (Section 2.2, steps 2-5;
// Alg. 1).  When a level's key space is small (2^(b(g-m)) keys, e.g.
// 4^6 = 4096 DNA 6-mers) every key can be a feature: F is dense, and all
// masks of a run of the level stack into one matrix A with a row per
// sequence and a column per (mask, key), so that C_m += A A^T.  No sort is
// needed: the scatter kernel counts A[x, (mask, key)] directly.
//
// Exactness.  A holds D0 = min(count, 16), which e4m3 represents exactly;
// products (<= 256) and partial sums are exact in the f32 accumulators
// while they stay within 2^24 - 1, so the GEMM closes an accumulation
// "round" and adds it into the int32 C every floor(cap / (128 maxD0^2))
// stages of 128 columns (cap = 2^24 - 1 unless a caller lowers it), maxD0
// being the largest D0 the scatter kernel wrote -- or once per macro tile
// when maxD0 times a row's largest possible sum (windows x masks) stays
// within cap, which bounds every partial sum.  The tests drive real partial
// sums of one round to just below 2^24 and compare with the oracle.  A
// count c > 16 is also appended to an overflow list, and the fix
// kernel adds the exact difference A A^T - D0 D0^T, which is nonzero only
// in rows and columns of overflowing sequences:
//   (x, y), y without overflow at the column:  (c_x - 16) D0(y)
//   (x, y), both overflowing at the column:    c_x c_y - 256
// (the second as (c_x-16) 16 + (c_y-16) 16 + (c_x-16)(c_y-16), one term
// from each entry's row scan and the product from the pair scan).
//
// GEMM structure.  One CTA per SM walks a list of macro tiles of 256 x 256
// outputs (upper triangle only: C is symmetric), each covering every mask
// run of its (dataset, level), so C receives one epilogue per macro tile.
// Warp 5 loads 128-column slices of A's rows I2*256.. (two 128-row blocks)
// and J2*256.. (256 rows) with TMA (128-byte swizzle) into a three-stage
// ring; one thread of warp 4 issues tcgen05.mma (M = 128, N = 256, K = 32)
// into two 256-column TMEM accumulators, one per 128-row half; warps 0-3
// read them back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and
// add the upper-triangle part into C.  Hand-offs use mbarriers.  Every
// wait is bounded: a timeout raises an error bit, stops every role, waits
// (bounded) for the copies and MMAs already issued, and frees tensor memory.
#include <cuda.h>  // CUtensorMap and its enums; the encoder is fetched at run time

#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "launch.h"

namespace gk {

namespace {

constexpr int kStages = 3;
constexpr uint32_t kSubBytes = 128 * 128;         // 128 rows x 128 e4m3 columns
constexpr uint32_t kStageBytes = 4 * kSubBytes;   // A rows I2*256 + {0, 128}, B rows J2*256 + {0, 128}
constexpr int kMmaWarp = 4, kTmaWarp = 5;
constexpr int kGemmThreads = 192;
constexpr uint32_t kTmemCols = 512;  // two 128 x 256 f32 accumulators
constexpr int kScatterThreads = 512;
constexpr int kScatterMasks = 16;  // masks of one scatter block held in shared memory
constexpr int kScatterWarps = kScatterThreads / 32;
constexpr int kScatterRuns = 5;    // kept-position runs of a mask cut in registers
constexpr int kRunMasks = 64;      // masks of one problem whose runs a scatter block stages
constexpr int kRowKeys = 1024;     // windows of a row whose 32-bit full keys a block stages

// A mask's kept-position runs for the scatter's 32-bit cut (nruns = ~0:
// the mask takes the generic cut).  A run moves from bit sr of the full key
// to bit sl <= sr of the masked key, so it is (full >> (sr - sl)) & (mask
// << sl): one shift and one AND-OR per run.
struct MaskRuns {
  uint32_t nruns;
  uint32_t sh[kScatterRuns], mk[kScatterRuns];
};
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s (drains; default for the role waits)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)(16 >> 4) << 16;          // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b))
               : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity.  Returns false when the
// wait ran out after `limit` cycles (and then raises the abort flag) or
// another role aborted.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile uint32_t* abort_flag,
                                         long long limit) {
  const long long t0 = clock64();
  for (;;) {
    if (bar_test(b, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag: used while unwinding, for work
// already issued.
__device__ __forceinline__ void bar_drain(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!bar_test(b, parity) && clock64() - t0 <= kWaitCycles) {
  }
}

__device__ __forceinline__ void tma_load(uint32_t dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"((uint64_t)tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Stages (128 columns each) per exact accumulation round, so that no
// partial sum of a round exceeds `cap` (at most 2^24 - 1, where f32 holds
// every integer).  Every partial sum of a (x, y) entry is at most
// sum_k A[x,k] A[y,k] <= maxc * sum_k A[y,k] <= maxc * wmasks (each window
// of y adds at most one to one column of each mask), so when that stays
// within `cap` the whole macro tile is one round; otherwise a stage adds at
// most 128 maxc^2.
__device__ __forceinline__ uint32_t stages_per_round(const uint32_t* maxc, uint32_t nk, uint32_t wmasks,
                                                     uint32_t cap) {
  const uint32_t mc = *(const volatile uint32_t*)maxc;
  if (mc == 0 || (wmasks != 0 && (uint64_t)mc * wmasks <= cap)) return nk > 0 ? nk : 1;
  uint64_t s = (uint64_t)cap / (128ull * mc * mc);
  if (s < 1) s = 1;
  return (uint32_t)(s < nk ? s : nk);
}

// Two 16-bit counts (each <= 16) -> two e4m3 bytes, low count in the low
// byte.  The counts become exact f16 values through the 1024-offset form
// (the f16 bits of 1024 + v are 0x6400 | v), then one hardware conversion
// packs both.
__device__ __forceinline__ uint32_t e4m3x2_of_counts(uint32_t clamped) {
  const uint32_t biased = clamped | 0x64006400u;
  uint32_t h;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(h) : "r"(biased), "r"(0x64006400u));
  uint16_t e;
  asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(e) : "r"(h));
  return e;
}

// e4m3 bytes of the counts 0..7 (1 = 0x38: exponent 7, mantissa 0; ...;
// 7 = 0x4E), as the eight bytes of a byte-permute table.
constexpr uint32_t kE4m3Counts0to3 = 0x44403800u;
constexpr uint32_t kE4m3Counts4to7 = 0x4E4C4A48u;

// Four counts 0..7, two per word with the lower column in the low half, ->
// their four e4m3 bytes in column order: the counts become the four 3-bit
// selectors of one byte permute over the table above.
__device__ __forceinline__ uint32_t e4m3x4_of_small_counts(uint32_t w01, uint32_t w23) {
  const uint32_t t = w01 | (w23 << 8);  // c0 at bit 0, c2 at 8, c1 at 16, c3 at 24
  return __byte_perm(kE4m3Counts0to3, kE4m3Counts4to7, t | (t >> 12));
}

// The integer an e4m3 byte of a count (0..16) encodes: exponent bias 7,
// three mantissa bits, v = 2^(e-7) (1 + m/8).
__device__ __forceinline__ uint32_t e4m3_small_value(uint32_t b) {
  if (b == 0) return 0;
  return ((8 + (b & 7)) << ((b >> 3) - 7)) >> 3;
}

}  // namespace

// Builds the rows of A: one block per row of the wave, walking the row's
// column chunks of kDenseScatterCols.  Counts are gathered in shared memory
// and each chunk is written out whole (zeros included), so A needs no
// separate clearing; padded rows come out all zero.  The conversion loop
// clears the counts it has read, ready for the next chunk.  kNarrow: the
// full g-mer keys have at most 32 bits (masked keys cut in 32-bit
// arithmetic).
template <bool kNarrow>
__global__ void __launch_bounds__(kScatterThreads, 3)
k_dense_scatter(const DenseProb* __restrict__ probs, uint32_t nprobs, uint32_t p0, const DsPack* __restrict__ dsp,
                const MaskDesc* __restrict__ masks, const uint64_t* __restrict__ fullkey, uint32_t* __restrict__ ovf_n,
                DenseOvf* __restrict__ ovf, uint32_t ovf_cap) {
  extern __shared__ uint32_t cnt[];  // two 16-bit counts per word (counts <= 65535 windows)
  __shared__ MaskDesc smask[kNarrow ? 1 : kScatterMasks];
  __shared__ MaskRuns sruns[kNarrow ? kRunMasks : 1];
  __shared__ uint32_t srow[kNarrow ? kRowKeys : 1];
  const uint32_t bx = blockIdx.x, tid = threadIdx.x;
  uint32_t lo = 0, hi = nprobs;  // last problem with row0 <= bx
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (probs[mid].row0 <= bx)
      lo = mid;
    else
      hi = mid;
  }
  const DenseProb& P = probs[lo];
  const uint64_t ld = P.ld;
  const uint32_t x = bx - P.row0;
  const uint32_t kb = P.key_bits;
  uint32_t w0 = 0, nw = 0;
  const uint64_t* fk = fullkey;
  if (x < P.n) {
    const DsPack& D = dsp[P.ds];
    w0 = D.woff[x];
    nw = D.woff[x + 1] - w0;
    fk = fullkey + D.win0 + w0;
  }
  {
    const uint32_t words = (uint32_t)(ld < (uint64_t)kDenseScatterCols ? ld : kDenseScatterCols) / 2;
    for (uint32_t i = tid; i < words / 4; i += kScatterThreads) ((uint4*)cnt)[i] = make_uint4(0, 0, 0, 0);
  }
  // 32-bit keys: the runs of every mask of the problem, and the row's full
  // keys, staged once (every chunk cuts the same keys).
  const bool keys_staged = kNarrow && nw <= (uint32_t)kRowKeys;
  if (keys_staged)
    for (uint32_t i = tid; i < nw; i += kScatterThreads) srow[i] = (uint32_t)fk[i];
  const bool runs_staged = kNarrow && P.mcount <= (uint32_t)kRunMasks;
  if (runs_staged) {
    for (uint32_t i = tid; i < P.mcount; i += kScatterThreads) {
      const MaskDesc& md = masks[P.mfirst + i];
      MaskRuns r{};
      r.nruns = (md.fold == 0 && md.nruns <= (uint32_t)kScatterRuns) ? md.nruns : ~0u;
#pragma unroll
      for (int q = 0; q < kScatterRuns; ++q) {
        const bool on = (uint32_t)q < md.nruns && r.nruns != ~0u;
        r.sh[q] = on ? md.sr[q] - md.sl[q] : 0u;
        r.mk[q] = on ? (uint32_t)md.msk[q] << md.sl[q] : 0u;
      }
      sruns[i] = r;
    }
  }
  uint32_t cmax = 0;  // per-half maximum of every count word
  for (uint64_t c0 = 0; c0 < ld; c0 += kDenseScatterCols) {
    const uint32_t ncol = (uint32_t)(ld - c0 < (uint64_t)kDenseScatterCols ? ld - c0 : kDenseScatterCols);
    const uint32_t mu0 = (uint32_t)(c0 >> kb);
    uint32_t mu1 = (uint32_t)((c0 + ncol - 1) >> kb) + 1;
    if (mu1 > P.mcount) mu1 = P.mcount;
    const uint32_t nmu = (nw > 0 && mu1 > mu0) ? mu1 - mu0 : 0;
    const bool staged = !kNarrow && nmu <= (uint32_t)kScatterMasks;
    if (staged) {
      // The chunk's masks, for warp-broadcast reads below.
      const uint32_t words = nmu * (uint32_t)(sizeof(MaskDesc) / 4);
      const uint32_t* src = (const uint32_t*)(masks + P.mfirst + mu0);
      for (uint32_t i = tid; i < words; i += kScatterThreads) ((uint32_t*)smask)[i] = src[i];
    }
    __syncthreads();
    if constexpr (kNarrow) {
      // Tasks of (mask, slice of the row's windows), one per warp at a time,
      // kScatterWarps of them per chunk when the chunk has that few masks: a
      // warp loads its mask's runs once (uniform shared-memory reads) and
      // walks its windows 32 at a time, cutting each key with shifts and
      // masks alone (runs mode; folded keys take the generic cut).
      const uint32_t S = nmu ? max(1u, (uint32_t)kScatterWarps / nmu) : 1u;
      const uint32_t per = ((nw + S - 1) / S + 31) & ~31u;
      for (uint32_t task = tid >> 5; task < nmu * S; task += kScatterWarps) {
        const uint32_t mi = task / S, s = task - mi * S;
        // Column of key 0 of the mask within the chunk, modulo 2^32 (a
        // problem's row holds fewer than 2^31 columns): keys of the masks
        // outside the chunk wrap to indices above ncol.
        const uint32_t cbase = ((mu0 + mi) << kb) - (uint32_t)c0;
        const uint32_t wlo = s * per, whi = min(nw, wlo + per);
        const uint32_t nr = runs_staged ? sruns[mu0 + mi].nruns : ~0u;
        if (nr != ~0u) {
          const MaskRuns& mr = sruns[mu0 + mi];
          uint32_t sh[kScatterRuns], mk[kScatterRuns];
#pragma unroll
          for (int r = 0; r < kScatterRuns; ++r) {
            sh[r] = mr.sh[r];
            mk[r] = mr.mk[r];
          }
          for (uint32_t wi = wlo + (tid & 31); wi < whi; wi += 32) {
            const uint32_t f = keys_staged ? srow[wi] : (uint32_t)fk[wi];
            uint32_t k = 0;
#pragma unroll
            for (int r = 0; r < kScatterRuns; ++r) k |= (f >> sh[r]) & mk[r];
            const uint32_t col = cbase + k;
            if (col < ncol) atomicAdd(&cnt[col >> 1], 1u << (16 * (col & 1)));
          }
        } else {
          const MaskDesc& md = masks[P.mfirst + mu0 + mi];
          for (uint32_t wi = wlo + (tid & 31); wi < whi; wi += 32) {
            const uint32_t col = cbase + masked_key32((uint32_t)fk[wi], md);
            if (col < ncol) atomicAdd(&cnt[col >> 1], 1u << (16 * (col & 1)));
          }
        }
      }
    } else {
      // 64-bit keys: mask-major over (mask, window), the lanes of a warp
      // mostly sharing one mask and reading consecutive windows.
      uint32_t mi = nw ? tid / nw : 0, w = nw ? tid - mi * nw : 0;
      for (uint32_t i = tid; i < nw * nmu; i += kScatterThreads) {
        const MaskDesc& md = staged ? smask[mi] : masks[P.mfirst + mu0 + mi];
        const uint64_t col = (((uint64_t)(mu0 + mi) << kb) | masked_key(fk[w], md)) - c0;
        if (col < ncol) atomicAdd(&cnt[col >> 1], 1u << (16 * (uint32_t)(col & 1)));
        w += kScatterThreads;
        while (w >= nw) {
          w -= nw;
          ++mi;
        }
      }
    }
    __syncthreads();
    // Eight columns (one 16-byte word of counts) per thread and step:
    // consecutive threads take consecutive words, so every shared-memory
    // access of a warp covers 512 contiguous bytes and every global store
    // 256 contiguous bytes.
    uint2* out = (uint2*)(P.A + (uint64_t)x * ld + c0);
    uint4* cw = (uint4*)cnt;
    auto convert = [&](uint32_t u, const uint4 a) {
      const uint32_t m = __vmaxu2(__vmaxu2(a.x, a.y), __vmaxu2(a.z, a.w));
      cmax = __vmaxu2(cmax, m);
      if ((m & 0xFFF8FFF8u) == 0u)  // every count <= 7 (nearly all words): table lookup
        return make_uint2(e4m3x4_of_small_counts(a.x, a.y), e4m3x4_of_small_counts(a.z, a.w));
      const uint32_t w[4] = {a.x, a.y, a.z, a.w};
      uint32_t e[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) e[q] = e4m3x2_of_counts(__vminu2(w[q], 0x00100010u));
      // A half h of m exceeds 16 iff h + 15 reaches bit 5 or h is above
      // 65520 (h + 15 then carries out of its half); both show in bits
      // 5-15 of (m + 15) | m.
      if ((((m + 0x000F000Fu) | m) & 0xFFE0FFE0u) != 0u) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t c = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
          if (c > 16) {
            const uint32_t slot = atomicAdd(ovf_n, 1u);
            if (slot < ovf_cap) ovf[slot] = DenseOvf{p0 + lo, x, (uint32_t)(c0 + 8 * u + q), c};
          }
        }
      }
      return make_uint2(e[0] | (e[1] << 16), e[2] | (e[3] << 16));
    };
    // Two words per thread and step (both reads in flight together).
    const uint32_t nwords = ncol / 8;
    uint32_t u = tid;
    for (; u + kScatterThreads < nwords; u += 2 * kScatterThreads) {
      const uint4 a = cw[u], b = cw[u + kScatterThreads];
      cw[u] = make_uint4(0, 0, 0, 0);
      cw[u + kScatterThreads] = make_uint4(0, 0, 0, 0);
      out[u] = convert(u, a);
      out[u + kScatterThreads] = convert(u + kScatterThreads, b);
    }
    if (u < nwords) {
      const uint4 a = cw[u];
      cw[u] = make_uint4(0, 0, 0, 0);
      out[u] = convert(u, a);
    }
    // The next chunk's counting waits at its first barrier for this
    // conversion (and its clearing) to finish.
  }
  uint32_t mymax = min(max(cmax & 0xFFFFu, cmax >> 16), 16u);  // the largest entry of A
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
  if ((tid & 31) == 0 && mymax) atomicMax(P.maxc, mymax);
}

// Exact correction for counts above 16 (see the top of this file): one warp
// per overflow entry scans the entry's column of A over every row, then the
// later entries of the list for the same (problem, column).
__global__ void __launch_bounds__(256)
k_dense_fix(const DenseProb* __restrict__ probs, const uint32_t* __restrict__ ovf_n, const DenseOvf* __restrict__ ovf,
            uint32_t ovf_cap, uint32_t* __restrict__ status) {
  const uint32_t E = *ovf_n;
  if (E > ovf_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kErrDenseOverflow);
    return;
  }
  const uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= E) return;
  const DenseOvf e = ovf[i];
  const DenseProb& P = probs[e.prob];
  const uint32_t n = P.n, x = e.x, d = e.count - 16;
  const uint8_t* colp = P.A + e.col;
  uint32_t* C = P.C;
  for (uint32_t y = lane; y < n; y += 32) {
    if (y == x) {
      atomicAdd(&C[(uint64_t)x * n + x], 32u * d + d * d);  // (16 + d)^2 - 16^2
      continue;
    }
    const uint32_t v = e4m3_small_value(colp[(uint64_t)y * P.ld]);
    if (v) {
      const uint32_t r = min(x, y), q = max(x, y);
      atomicAdd(&C[(uint64_t)r * n + q], d * v);
    }
  }
  for (uint32_t j = i + 1 + lane; j < E; j += 32) {
    const DenseOvf f = ovf[j];
    if (f.prob == e.prob && f.col == e.col) {
      const uint32_t r = min(x, f.x), q = max(x, f.x);
      atomicAdd(&C[(uint64_t)r * n + q], d * (f.count - 16));
    }
  }
}

// Row halves a of macro tile (I2, J2) that hold rows below n: bit a set
// when rows I2*256+128a.. start below n.
__device__ __forceinline__ uint32_t row_halves(uint32_t I2, uint32_t n) {
  return (I2 * 256 < n ? 1u : 0u) | (I2 * 256 + 128 < n ? 2u : 0u);
}

__global__ void __launch_bounds__(kGemmThreads, 1)
k_dense_gemm(const DenseProb* __restrict__ probs, const uint32_t* __restrict__ tiles, uint32_t ntiles,
             uint32_t sum_cap, long long wait_cycles, uint32_t* __restrict__ status) {
  extern __shared__ uint8_t raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], tfull, tempty, done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile uint32_t abort_flag;
  uint8_t* sm = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full_bar[s], 1);
      bar_init(&empty_bar[s], 1);
    }
    bar_init(&tfull, 1);
    bar_init(&tempty, 128);
    bar_init(&done_bar, 1);
    abort_flag = 0;
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tmem_base;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      uint32_t it = 0;
      bool stop = false;
      for (uint32_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const uint32_t* tl = tiles + kDenseTileWords * t;
        const uint32_t pa = tl[0], pn = tl[1], I2 = tl[2], J2 = tl[3], s0 = tl[4], s1 = tl[5];
        const uint32_t st = row_halves(I2, probs[pa].n);
        const bool needA[2] = {(st & 1u) != 0, (st & 2u) != 0};
        const uint32_t bytes = kSubBytes * (2 + needA[0] + needA[1]);  // B: both 128-row blocks
        uint32_t g = 0;  // the run's stages before problem p
        for (uint32_t p = pa; p < pa + pn && !stop && g < s1; ++p) {
          const void* tm = probs[p].tmap;
          const uint32_t nk = (uint32_t)(probs[p].ld / 128);
          const uint32_t k0 = s0 > g ? min(s0 - g, nk) : 0u, k1 = min(nk, s1 - g);
          g += nk;
          for (uint32_t k = k0; k < k1; ++k, ++it) {
            const uint32_t s = it % kStages;
            if (!bar_wait(&empty_bar[s], ((it / kStages) & 1) ^ 1, &abort_flag, wait_cycles)) {
              stop = true;
              break;
            }
            const uint32_t dst = smem_u32(sm + s * kStageBytes);
            bar_expect_tx(&full_bar[s], bytes);
#pragma unroll
            for (uint32_t a = 0; a < 2; ++a)
              if (needA[a]) tma_load(dst + a * kSubBytes, tm, (int)(k * 128), (int)(I2 * 256 + a * 128), &full_bar[s]);
#pragma unroll
            for (uint32_t b = 0; b < 2; ++b)
              tma_load(dst + (2 + b) * kSubBytes, tm, (int)(k * 128), (int)(J2 * 256 + b * 128), &full_bar[s]);
          }
        }
      }
      // Let the copies already issued land before the block can exit.
      for (uint32_t s = 0; s < (uint32_t)kStages; ++s)
        if (it > s) {
          const uint32_t j = s + kStages * ((it - 1 - s) / kStages);
          bar_drain(&full_bar[s], (j / kStages) & 1);
        }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // f32 accumulator, e4m3 A and B (type code 0), K-major, N = 256, M = 128.
      const uint32_t idesc = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
      uint32_t it = 0, round = 0;
      bool stop = false;
      for (uint32_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const uint32_t* tl = tiles + kDenseTileWords * t;
        const uint32_t pa = tl[0], pn = tl[1], I2 = tl[2], s0 = tl[4], s1 = tl[5];
        const uint32_t st = row_halves(I2, probs[pa].n);
        uint32_t total = 0;
        for (uint32_t p = pa; p < pa + pn; ++p) total += (uint32_t)(probs[p].ld / 128);
        const uint32_t lo = min(s0, total), hi = min(s1, total);
        const uint32_t spr = stages_per_round(probs[pa].maxc, hi - lo, probs[pa].wmasks, sum_cap);
        uint32_t kr = 0;  // stages into the current round
        uint32_t g = 0;   // the run's stages before problem p
        for (uint32_t p = pa; p < pa + pn && !stop && g < hi; ++p) {
          const uint32_t nk = (uint32_t)(probs[p].ld / 128);
          const uint32_t k0 = lo > g ? min(lo - g, nk) : 0u, k1 = min(nk, hi - g);
          g += nk;
          for (uint32_t k = k0; k < k1; ++k, ++it) {
            if (kr == 0) {
              if (!bar_wait(&tempty, (round & 1) ^ 1, &abort_flag, wait_cycles)) {
                stop = true;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
            }
            const uint32_t s = it % kStages;
            if (!bar_wait(&full_bar[s], (it / kStages) & 1, &abort_flag, wait_cycles)) {
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = smem_u32(sm + s * kStageBytes);
#pragma unroll
            for (uint32_t ah = 0; ah < 2; ++ah) {
              if (!(st & (1u << ah))) continue;
              const uint32_t a0 = base + ah * kSubBytes, b0 = base + 2 * kSubBytes;
              const uint32_t d = taddr + 256 * ah;
#pragma unroll
              for (uint32_t j = 0; j < 4; ++j) {
                const uint32_t acc = (kr > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                    "l"(smem_desc(a0 + j * 32)), "l"(smem_desc(b0 + j * 32)), "r"(idesc), "r"(acc));
              }
            }
            mma_commit(&empty_bar[s]);
            if (++kr == spr) {
              mma_commit(&tfull);
              ++round;
              kr = 0;
            }
          }
        }
        if (!stop && kr > 0) {
          mma_commit(&tfull);
          ++round;
        }
      }
      // Every MMA issued must finish before tensor memory is freed.
      mma_commit(&done_bar);
      bar_drain(&done_bar, 0);
    }
  } else {
    // Epilogue warps 0-3: TMEM lanes 32*warp.. = rows of each sub-tile.
    uint32_t round = 0;
    bool stop = false;
    for (uint32_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const uint32_t* tl = tiles + kDenseTileWords * t;
      const uint32_t pa = tl[0], pn = tl[1], I2 = tl[2], J2 = tl[3], s0 = tl[4], s1 = tl[5];
      const uint32_t n = probs[pa].n;
      const uint32_t st = row_halves(I2, n);
      uint32_t total = 0;
      for (uint32_t p = pa; p < pa + pn; ++p) total += (uint32_t)(probs[p].ld / 128);
      const uint32_t lo = min(s0, total), hi = min(s1, total);
      const uint32_t spr = stages_per_round(probs[pa].maxc, hi - lo, probs[pa].wmasks, sum_cap);
      const uint32_t nr = (hi - lo + spr - 1) / spr;
      // One round, the whole run and no other writer: the tile's C entries
      // are still zero, so plain (vector) stores replace the atomic adds.
      const bool store = nr == 1 && probs[pa].sole != 0 && lo == 0 && hi == total;
      uint32_t* C = probs[pa].C;
      for (uint32_t r = 0; r < nr; ++r, ++round) {
        if (!__all_sync(0xffffffffu, bar_wait(&tfull, round & 1, &abort_flag, wait_cycles))) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (uint32_t ah = 0; ah < 2; ++ah) {
          if (!(st & (1u << ah))) continue;
          const uint32_t row = I2 * 256 + ah * 128 + warp * 32 + lane;
          const uint32_t col0 = J2 * 256;
          uint32_t* crow = C + (uint64_t)row * n;
#pragma unroll 1
          for (uint32_t cb = 0; cb < 256; cb += 32) {
            uint32_t v[32];
            const uint32_t a = taddr + 256 * ah + cb + ((warp * 32) << 16);
            __syncwarp();
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(a));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < n) {
              const uint32_t c0 = col0 + cb;
              uint32_t* dst = crow + c0;
              if (!store) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                  const uint32_t val = (uint32_t)__uint_as_float(v[j]);
                  if (c0 + j < n && c0 + j >= row && val) atomicAdd(&dst[j], val);
                }
              } else if (c0 >= row && c0 + 32 <= n && ((uintptr_t)dst & 15u) == 0) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                  *(uint4*)(dst + j) = make_uint4((uint32_t)__uint_as_float(v[j]), (uint32_t)__uint_as_float(v[j + 1]),
                                                  (uint32_t)__uint_as_float(v[j + 2]), (uint32_t)__uint_as_float(v[j + 3]));
              } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (c0 + j < n && c0 + j >= row) dst[j] = (uint32_t)__uint_as_float(v[j]);
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        bar_arrive(&tempty);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (tid == 0 && abort_flag) atomicOr(status, kErrTimeout);
  if (warp == kMmaWarp) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols));
  }
}

// ------------------------------------------------------- heavy features --

// One block per tile of a run-length chunk, over the tile's range of the
// segment's entries.  A feature starts at entry e when e = 0 or the
// previous entry's feature end differs (all entries of a feature share
// it); a warp checks its 32 entries, then examines each qualifying start
// together (the largest count of the feature must be <= 16, so that A
// holds the counts exactly).
__global__ void __launch_bounds__(256)
k_heavy_mark(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
             const uint32_t* __restrict__ segtot, const uint32_t* __restrict__ mask_level,
             const uint32_t* __restrict__ hmap, uint32_t levels, const HeavyProb* __restrict__ hprobs,
             const uint32_t* __restrict__ eseq, const uint32_t* __restrict__ efe,
             HeavyItem* __restrict__ items, uint32_t* __restrict__ nitems) {
  const uint32_t t = blockIdx.x;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t hp = hmap[sd.ds * levels + mask_level[sd.mask]];
  if (hp == kNone) return;
  const HeavyProb& H = hprobs[hp];
  const uint32_t E = segtot[2 * (uint64_t)s];
  const uint64_t e_beg = (uint64_t)(t - sd.tile0) * kTile;
  if (e_beg >= E) return;
  const uint32_t e_end = (uint32_t)min((uint64_t)E, e_beg + kTile);
  const uint32_t* __restrict__ es = eseq + sd.pool;
  const uint32_t* __restrict__ ef = efe + sd.pool;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t b = (uint32_t)e_beg + w * 32; b < e_end; b += blockDim.x) {
    const uint32_t e = b + lane;
    uint32_t fe = 0;
    bool cand = false;
    if (e < e_end) {
      fe = ef[e];
      cand = (e == 0 || ef[e - 1] != fe) && fe > e && fe <= E && fe - e >= H.T;
    }
    uint32_t bm = __ballot_sync(0xffffffffu, cand);
    while (bm) {
      const int L0 = __ffs(bm) - 1;
      bm &= bm - 1;
      const uint32_t e0 = __shfl_sync(0xffffffffu, e, L0), f0 = __shfl_sync(0xffffffffu, fe, L0);
      uint32_t mx = 0;
      for (uint32_t q = e0 + lane; q < f0; q += 32) mx = max(mx, es[q] & 0xFFFFu);
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (mx <= 16 && lane == 0) {
        const uint32_t col = atomicAdd(H.ncols, 1u);
        if (col < H.cap) {
          const uint32_t slot = atomicAdd(nitems, 1u);
          items[slot] = HeavyItem{sd.pool, e0, f0 - e0, col, hp, {0u, 0u}};
          atomicMax(H.maxc, mx);
        }
      }
    }
  }
}

// Grid (rows, problems): clears the used columns of one row of A.
__global__ void __launch_bounds__(256)
k_heavy_zero(const HeavyProb* __restrict__ hprobs, DenseProb* __restrict__ dprobs,
             unsigned long long* __restrict__ work) {
  const uint32_t hp = blockIdx.y, row = blockIdx.x;
  const HeavyProb& H = hprobs[hp];
  if (row >= H.n_pad) return;
  const uint32_t used = min(*H.ncols, H.cap);
  const uint32_t K = (used + 127u) & ~127u;
  uint4* a = (uint4*)(H.A + (uint64_t)row * H.stride);
  for (uint32_t i = threadIdx.x; i < K / 16; i += blockDim.x) a[i] = make_uint4(0u, 0u, 0u, 0u);
  if (row == 0 && threadIdx.x == 0) {
    dprobs[H.prob].ld = K;
    atomicAdd(&work[0], (unsigned long long)used);
    atomicAdd(&work[1], (unsigned long long)used * H.n * (H.n + 1ull));
  }
}

// One warp per listed feature.
__global__ void __launch_bounds__(256)
k_heavy_scatter(const HeavyProb* __restrict__ hprobs, const HeavyItem* __restrict__ items,
                const uint32_t* __restrict__ nitems, const uint32_t* __restrict__ eseq,
                uint32_t* __restrict__ efe) {
  const uint32_t N = *nitems;
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t i = blockIdx.x * 8 + (threadIdx.x >> 5); i < N; i += gridDim.x * 8) {
    const HeavyItem it = items[i];
    const HeavyProb& H = hprobs[it.hp];
    const uint32_t* __restrict__ es = eseq + it.pool;
    uint32_t* __restrict__ ef = efe + it.pool;
    for (uint32_t q = it.fs + lane; q < it.fs + it.L; q += 32) {
      const uint32_t v = es[q];
      H.A[(uint64_t)(v >> 16) * H.stride + it.col] = (uint8_t)e4m3x2_of_counts(v & 0xFFFFu);
      ef[q] |= kHeavyBit;
    }
  }
}

void launch_heavy_mark(const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                       const uint32_t* segtot, const uint32_t* mask_level, const uint32_t* hmap,
                       uint32_t levels, const HeavyProb* hprobs, const uint32_t* eseq,
                       const uint32_t* efe, HeavyItem* items, uint32_t* nitems, cudaStream_t st) {
  if (ntiles == 0) return;
  k_heavy_mark<<<ntiles, 256, 0, st>>>(segs, tile_seg, segtot, mask_level, hmap, levels, hprobs, eseq, efe,
                                       items, nitems);
}

void launch_heavy_zero(const HeavyProb* hprobs, uint32_t nh, uint32_t max_rows, DenseProb* dprobs,
                       unsigned long long* work, cudaStream_t st) {
  if (nh == 0 || max_rows == 0) return;
  k_heavy_zero<<<dim3(max_rows, nh), 256, 0, st>>>(hprobs, dprobs, work);
}

void launch_heavy_scatter(const HeavyProb* hprobs, const HeavyItem* items, const uint32_t* nitems,
                          uint32_t* eseq, uint32_t* efe, int nsm, cudaStream_t st) {
  k_heavy_scatter<<<nsm * 4, 256, 0, st>>>(hprobs, items, nitems, eseq, efe);
}

size_t dense_scatter_smem() { return (size_t)kDenseScatterCols * 2; }
size_t dense_gemm_smem() { return (size_t)kStages * kStageBytes + 1024; }

int dense_init() {
  cudaError_t e = cudaFuncSetAttribute(k_dense_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dense_gemm_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dense_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dense_scatter_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dense_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dense_scatter_smem());
  return (int)e;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  return fn;
}

}  // namespace

int dense_encode_tmap(void* out, void* A, uint64_t ld, uint64_t rows) {
  static_assert(sizeof(CUtensorMap) == kDenseTmapBytes, "tensor map size");
  EncodeTiledFn fn = encoder();
  if (!fn) return -1;
  const cuuint64_t dims[2] = {ld, rows};
  const cuuint64_t strides[1] = {ld};
  const cuuint32_t box[2] = {128, 128};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn((CUtensorMap*)out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, A, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

void launch_dense_scatter(const DenseProb* d_probs, uint32_t nprobs, uint32_t p0, uint32_t rows,
                          const DsPack* dsp, const MaskDesc* masks, const uint64_t* fullkey,
                          uint32_t full_bits, uint32_t* ovf_n, DenseOvf* ovf, uint32_t ovf_cap,
                          cudaStream_t st) {
  if (nprobs == 0 || rows == 0) return;
  if (full_bits <= 32)
    k_dense_scatter<true><<<rows, kScatterThreads, dense_scatter_smem(), st>>>(
        d_probs, nprobs, p0, dsp, masks, fullkey, ovf_n, ovf, ovf_cap);
  else
    k_dense_scatter<false><<<rows, kScatterThreads, dense_scatter_smem(), st>>>(
        d_probs, nprobs, p0, dsp, masks, fullkey, ovf_n, ovf, ovf_cap);
}

void launch_dense_fix(const DenseProb* d_probs, const uint32_t* ovf_n, const DenseOvf* ovf, uint32_t ovf_cap,
                      uint32_t* status, cudaStream_t st) {
  const uint32_t blocks = (ovf_cap + 7) / 8;
  k_dense_fix<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(d_probs, ovf_n, ovf, ovf_cap, status);
}

void launch_dense_gemm(const DenseProb* d_probs, const uint32_t* d_tiles, uint32_t ntiles, int nsm,
                       uint32_t sum_cap, long long wait_cycles, uint32_t* status, cudaStream_t st) {
  if (ntiles == 0) return;
  const uint32_t grid = ntiles < (uint32_t)nsm ? ntiles : (uint32_t)nsm;
  if (sum_cap == 0 || sum_cap > kDenseExactSum) sum_cap = kDenseExactSum;
  if (wait_cycles <= 0) wait_cycles = kWaitCycles;
  k_dense_gemm<<<grid, kGemmThreads, dense_gemm_smem(), st>>>(d_probs, d_tiles, ntiles, sum_cap, wait_cycles,
                                                                status);
}

}  // namespace gk
