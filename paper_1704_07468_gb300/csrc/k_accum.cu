// Kernel-update stage (Section 2.2, steps 2-5; Alg. 1 countAndUpdate and
// the sum C_m = sum_i C_m^i), inclusion-exclusion (Eq. 9), the kernel
// K = sum_m h_m N_m (Eq. 6, Eq. 7) and normalisation.
//
// For one mask, let F be the count matrix with F[f, x] = number of windows
// of sequence x whose (g-m)-mer is feature f.  The mask adds F^T F to C_m:
// for every feature, c_x * c_y to every pair of sequences holding it.  Only
// features held by several sequences touch off-diagonal entries (the paper
// counts those, "> 1", at step 2).
//
// k_accum accumulates rows of C_m in shared memory.  A work item is one row
// x of one dataset, one level m and a group of that level's masks; its
// warps walk the group's masks over the windows of x, and for each entry
// (f, x, c_x) of the row add c_x * c_y for every entry (f, y, c_y) of the
// same feature with y >= x.  Entries of a feature are sorted by sequence,
// so y >= x is the tail of the feature's entry range.  A window slot
// tagged as a one-sequence feature (kSingleTag | count) only adds count^2
// to the diagonal: summed in registers with the diagonal pairs of the other
// features, added once per item.  The row is then
// added to the global C_m with coalesced reductions.  Entries of heavy
// features (kHeavyBit in their feature end) are skipped: the tensor cores
// add those features' pairs.  Items are handed out
// group by group, so the rows being processed at any moment read the same
// few masks' entry arrays, which stay in L2.
#include <cstdint>

#include "common.cuh"
#include "launch.h"

namespace gk {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
// Entry ranges at least this long are walked by a whole warp, one range at
// a time; shorter ones by the variant's rounds.  The OR-owner rounds fill
// every lane, so variant 1 keeps ranges up to 63 in them (measured on DNA:
// threshold 32 / 64 / 128 / none: 10.74 / 10.37 / 10.78 / 10.88 ms).
constexpr uint32_t long_threshold(int variant) { return variant == 1 ? 64u : 32u; }

// 1 << d, and 0 for d >= 32 (PTX clamps the shift amount at the width).
__device__ __forceinline__ uint32_t bit_or_zero(uint32_t d) {
  uint32_t b;
  asm("shl.b32 %0, %1, %2;" : "=r"(b) : "r"(1u), "r"(d));
  return b;
}

// First entry in [lo, hi) whose sequence is >= seq.
__device__ __forceinline__ uint32_t lower_bound_seq(const uint32_t* __restrict__ es,
                                                    uint32_t lo, uint32_t hi,
                                                    uint32_t seq) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((es[mid] >> 16) < seq)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Eq. 9 then Eq. 7 for one (x, y): N_m = C_m - sum_{j<m} C(g-j, m-j) N_j,
// K = sum_m h_m N_m.  Arithmetic is modulo 2^32; every final N_m lies in
// [0, W_x W_y] and K < 2^31 (checked on the host), so the results are exact.
template <int kL = kMaxLevels>
__device__ __forceinline__ uint32_t ie_combine(const uint32_t* C, uint32_t M,
                                               const uint32_t (*ie)[kMaxLevels],
                                               const uint32_t* h,
                                               uint32_t* N) {
  uint32_t K = 0;
#pragma unroll
  for (int m = 0; m < kL; ++m) {
    if ((uint32_t)m <= M) {
      uint32_t v = C[m];
#pragma unroll
      for (int j = 0; j < m; ++j) v -= ie[m][j] * N[j];
      N[m] = v;
      K += h[m] * v;
    }
  }
  return K;
}

// kExpand chooses how a warp walks the entry ranges shorter than kLong
// (results are identical; the autotuner picks per workload):
//   0: up to four pairs per lane directly (each lane loads its own range),
//      the rest in rounds of 32 pairs whose owner lanes are found by a
//      shuffle binary search over the ranges' running counts;
//   1: every pair of a range shorter than 64 in rounds of 32 (consecutive
//      lanes load consecutive entries), owners found from a warp-wide OR of
//      the range starts that fall in the round (no shuffles; the owners'
//      data in a per-warp shared table);
//   2: the direct step of 0, then the rounds of 1 for what is left.
// Every variant is held to 32 registers, so that eight 256-thread blocks
// stay resident per SM.
template <int kThreads, int kExpand>
__global__ void __launch_bounds__(kThreads, 2048 / kThreads)
k_accum(const AccParams p) {
  constexpr uint32_t kLong = long_threshold(kExpand);
  extern __shared__ uint32_t acc[];   // ncols counters of one row of C_m + a trash slot
  __shared__ uint32_t s_item;
  constexpr int kWarps = kThreads / 32;
  // Per warp: the chunk's non-empty entry ranges in lane order (first entry
  // minus the range's first pair number, and the multiplier c_x).
  __shared__ uint2 s_rbc[kWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(p.counter, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= p.nitems) return;
    const uint32_t* I = p.items + (uint64_t)it * kItemWords;
    const uint32_t d = I[0], lvl = I[1], mfirst = I[2], mcount = I[3];
    const uint32_t x = I[4], c0 = I[5], c1 = I[6];
    const DsInfo ds = p.ds[d];
    const uint32_t width = c1 - c0;
    for (uint32_t i = threadIdx.x; i <= width; i += kThreads) acc[i] = 0;
    __syncthreads();
    const uint32_t wbeg = ds.woff[x], wend = ds.woff[x + 1];
    const uint32_t gd = ds.woff[ds.n];  // windows of the dataset: bound of every entry index
    const bool lo_cut = c0 > x, hi_cut = c1 < ds.n;
    const uint32_t nch = (wend - wbeg + 31) / 32;
    uint32_t n_pairs = 0, n_ent = 0;    // work counters of this thread
    uint32_t dsum = 0;                  // diagonal from one-sequence features
    for (uint32_t ch = w; ch < mcount * nch; ch += kWarps) {
      const uint32_t mu = mfirst + ch / nch;
      const uint32_t wi = wbeg + (ch % nch) * 32 + lane;
      const uint64_t pool = (uint64_t)mu * p.gtot + ds.win0;
      const uint32_t* __restrict__ ew = p.ewin + pool;
      const uint32_t* __restrict__ es = p.eseq + pool;
      const uint32_t* __restrict__ ef = p.efe + pool;
      uint32_t e = wi < wend ? ew[wi] : kNone;
      if (is_single(e)) {
        const uint32_t cs = e & 0xFFFFu;
        dsum += cs * cs;
        ++n_pairs;
        ++n_ent;
        e = kNone;
      }
      uint32_t lo = 0, cnt = 0, c = 0;
      if (e != kNone) {
        const uint32_t hi0 = e < gd ? ef[e] : 0;
        if (hi0 & kHeavyBit) {
          e = kNone;  // a heavy feature: the dense contraction adds its pairs
        } else if (e >= gd || hi0 > gd || hi0 <= e) {
          atomicOr(p.status, kErrBadEntry);  // corrupt entry: skip it
          e = kNone;
        } else {
          c = es[e] & 0xFFFFu;
          uint32_t hi = hi0;
          lo = e;
          if (lo_cut) lo = lower_bound_seq(es, e, hi, c0);
          if (hi_cut) hi = lower_bound_seq(es, lo, hi, c1);
          cnt = hi - lo;
        }
      }
      n_pairs += cnt;
      n_ent += e != kNone;
      // The range starts at x's own entry (the diagonal pair) unless the
      // item's columns begin after x.  Every lane of the chunk would add it
      // to the same counter acc[x] in one instruction; sum c^2 in
      // registers instead.
      if (e != kNone && lo == e && cnt > 0) {
        dsum += c * c;
        ++lo;
        --cnt;
      }
      // Long entry ranges: the whole warp walks one range at a time, lanes on
      // consecutive entries (every atomic instruction fully populated), four
      // loads in flight per lane.  Column indices are clamped to the trash
      // slot acc[width]; anything landing there is reported after the item.
      uint32_t longm = __ballot_sync(kFull, cnt >= kLong);
      while (longm) {
        const int L = __ffs(longm) - 1;
        longm &= longm - 1;
        const uint32_t lL = __shfl_sync(kFull, lo, L);
        const uint32_t nL = __shfl_sync(kFull, cnt, L);
        const uint32_t cL = __shfl_sync(kFull, c, L);
        const uint32_t* __restrict__ src = es + lL;
        for (uint32_t q = lane; q < nL; q += 128) {
          uint32_t v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = q + 32 * u < nL ? src[q + 32 * u] : 0u;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q + 32 * u < nL) atomicAdd(&acc[min((v[u] >> 16) - c0, width)], cL * (v[u] & 0xFFFFu));
        }
      }
      if (cnt >= kLong) cnt = 0;
      if constexpr (kExpand != 1) {
        // Short ranges: up to four pairs per lane directly.
        const uint32_t s4 = min(cnt, 4u);
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (uint32_t)u < s4 ? es[lo + u] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((uint32_t)u < s4) atomicAdd(&acc[min((v[u] >> 16) - c0, width)], c * (v[u] & 0xFFFFu));
        lo += s4;
        cnt -= s4;
      }
      if constexpr (kExpand == 0) {
        // The rest of the ranges in rounds of 32 pairs; the owner lane of a
        // pair is the first lane whose inclusive count exceeds it.
        if (__any_sync(kFull, cnt != 0)) {
          uint32_t incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
          }
          const uint32_t total = __shfl_sync(kFull, incl, 31);
          const uint32_t excl = incl - cnt;
          uint32_t p0 = 0;
          // Two full rounds at a time: both owner searches, then both entry
          // loads in flight before either atomic.
          for (; p0 + 64 <= total; p0 += 64) {
            const uint32_t pa = p0 + lane, pb = pa + 32;
            uint32_t oa = 0, ob = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
              const uint32_t ta = __shfl_sync(kFull, incl, oa + step - 1);
              const uint32_t tb = __shfl_sync(kFull, incl, ob + step - 1);
              if (ta <= pa) oa += step;
              if (tb <= pb) ob += step;
            }
            const uint32_t la = __shfl_sync(kFull, lo, oa) - __shfl_sync(kFull, excl, oa);
            const uint32_t lb = __shfl_sync(kFull, lo, ob) - __shfl_sync(kFull, excl, ob);
            const uint32_t ca = __shfl_sync(kFull, c, oa), cb = __shfl_sync(kFull, c, ob);
            const uint32_t va = es[la + pa], vb = es[lb + pb];
            atomicAdd(&acc[min((va >> 16) - c0, width)], ca * (va & 0xFFFFu));
            atomicAdd(&acc[min((vb >> 16) - c0, width)], cb * (vb & 0xFFFFu));
          }
          for (; p0 < total; p0 += 32) {
            const uint32_t pp = p0 + lane;
            uint32_t o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
              const uint32_t t = __shfl_sync(kFull, incl, o + step - 1);
              if (t <= pp) o += step;
            }
            const uint32_t lo_o = __shfl_sync(kFull, lo, o);
            const uint32_t ex_o = __shfl_sync(kFull, excl, o);
            const uint32_t c_o = __shfl_sync(kFull, c, o);
            if (pp < total) {
              const uint32_t v = es[lo_o + (pp - ex_o)];
              atomicAdd(&acc[min((v >> 16) - c0, width)], c_o * (v & 0xFFFFu));
            }
          }
        }
      } else {
        // Rounds of 32 pairs: round r gives lane i pair 32 r + i of the
        // ranges laid end to end, so consecutive lanes load consecutive
        // entries.  The ranges starting inside a round set one bit each in
        // a warp-wide OR; a pair's owner is the round's first owner plus
        // the starts at or before the pair.
        const uint32_t nz = __ballot_sync(kFull, cnt != 0);
        if (nz) {
          uint32_t incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
          }
          const uint32_t total = __shfl_sync(kFull, incl, 31);
          const uint32_t start = incl - cnt;  // the range's first pair number
          if (cnt) {
            const uint32_t rank = __popc(nz & lt_mask);
            s_rbc[w][rank] = make_uint2(lo - start, c);
          }
          __syncwarp();
          // Round p0 sets bit start - p0 - 1 for every range starting at
          // pairs p0 + 1 .. p0 + 32; empty ranges never set one.
          const uint32_t dpos = cnt ? start - 1u : 0x80000000u;
          uint32_t owner0 = 0;  // rank of the range holding the round's first pair
          uint32_t pp = lane;   // this lane's pair in the round
          const uint32_t full = total & ~31u;
          uint32_t p0 = 0;
          // Four rounds at a time: every entry load in flight before the atomics.
          for (; p0 + 96 < full; p0 += 128, pp += 128) {
            uint32_t bits[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) bits[q] = __reduce_or_sync(kFull, bit_or_zero(dpos - p0 - 32u * q));
            uint2 rc[4];
            uint32_t v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              rc[q] = s_rbc[w][owner0 + __popc(bits[q] & lt_mask)];
              owner0 += __popc(bits[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = es[rc[q].x + pp + 32u * q];
#pragma unroll
            for (int q = 0; q < 4; ++q) atomicAdd(&acc[min((v[q] >> 16) - c0, width)], rc[q].y * (v[q] & 0xFFFFu));
          }
          // Two rounds at a time: both entry loads are in flight before
          // either round's atomic.
          for (; p0 + 32 < full; p0 += 64, pp += 64) {
            const uint32_t bits0 = __reduce_or_sync(kFull, bit_or_zero(dpos - p0));
            const uint32_t bits1 = __reduce_or_sync(kFull, bit_or_zero(dpos - p0 - 32u));
            const uint32_t o1 = owner0 + __popc(bits0);
            const uint2 rc0 = s_rbc[w][owner0 + __popc(bits0 & lt_mask)];
            const uint2 rc1 = s_rbc[w][o1 + __popc(bits1 & lt_mask)];
            const uint32_t v0 = es[rc0.x + pp];
            const uint32_t v1 = es[rc1.x + pp + 32u];
            atomicAdd(&acc[min((v0 >> 16) - c0, width)], rc0.y * (v0 & 0xFFFFu));
            atomicAdd(&acc[min((v1 >> 16) - c0, width)], rc1.y * (v1 & 0xFFFFu));
            owner0 = o1 + __popc(bits1);
          }
          if (p0 < full) {
            const uint32_t bits = __reduce_or_sync(kFull, bit_or_zero(dpos - p0));
            const uint2 rc = s_rbc[w][owner0 + __popc(bits & lt_mask)];
            const uint32_t v = es[rc.x + pp];
            atomicAdd(&acc[min((v >> 16) - c0, width)], rc.y * (v & 0xFFFFu));
            owner0 += __popc(bits);
            pp += 32;
          }
          if (full < total) {
            const uint32_t bits = __reduce_or_sync(kFull, bit_or_zero(dpos - full));
            if (pp < total) {
              const uint2 rc = s_rbc[w][owner0 + __popc(bits & lt_mask)];
              const uint32_t v = es[rc.x + pp];
              atomicAdd(&acc[min((v >> 16) - c0, width)], rc.y * (v & 0xFFFFu));
            }
          }
          __syncwarp();
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
    if (lane == 0 && dsum && x >= c0 && x < c1) atomicAdd(&acc[x - c0], dsum);
    if (p.work) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        n_pairs += __shfl_xor_sync(kFull, n_pairs, o);
        n_ent += __shfl_xor_sync(kFull, n_ent, o);
      }
      if (lane == 0) {
        atomicAdd(&p.work[0], (unsigned long long)n_pairs);
        atomicAdd(&p.work[1], (unsigned long long)n_ent);
        if (w == 0) atomicAdd(&p.work[2], (unsigned long long)(wend - wbeg) * mcount);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && acc[width] != 0) atomicOr(p.status, kErrBadEntry);
    // Add the row into the global C_m (other groups of the level add to the
    // same row, possibly at the same time).
    uint32_t* __restrict__ crow = ds.C + ((uint64_t)lvl * ds.n + x) * ds.n + c0;
    for (uint32_t i = threadIdx.x; i < width; i += kThreads) {
      const uint32_t v = acc[i];
      if (v) atomicAdd(&crow[i], v);
    }
  }
}

// K(x, x) from the diagonal of C_0..C_M and r_x = 1 / sqrt(K(x, x)) (0
// when K(x, x) = 0) for normalisation.
__global__ void __launch_bounds__(256)
k_diag(const DsInfo* __restrict__ dsv, uint32_t nds, uint32_t nseq, const AccParams p) {
  const uint32_t gs = blockIdx.x * blockDim.x + threadIdx.x;
  if (gs >= nseq) return;
  uint32_t d = 0;
  while (d + 1 < nds && dsv[d + 1].seq0 <= gs) ++d;
  const DsInfo D = dsv[d];
  const uint32_t x = gs - D.seq0;
  const uint64_t nn = (uint64_t)D.n * D.n;
  const uint64_t o = (uint64_t)x * D.n + x;
  uint32_t C[kMaxLevels], N[kMaxLevels];
#pragma unroll
  for (int m = 0; m < kMaxLevels; ++m) C[m] = (uint32_t)m <= p.M ? D.C[m * nn + o] : 0u;
  const uint32_t K = ie_combine(C, p.M, p.ie, p.h, N);
  D.rinv[x] = K ? 1.0 / sqrt((double)K) : 0.0;
}

// Eq. 9 and Eq. 7 on the upper triangle of C, tile by tile, writing K, N_m
// and Khat at (x, y) and, through a shared-memory transpose, at (y, x).
// Khat(x, y) = (K * r_x) * r_y (a few ulp from K / sqrt(Kxx Kyy)), exactly
// 1 on a nonzero diagonal, 0 where a diagonal is 0.  Lower tiles exit.
// kL >= M + 1 bounds the levels held in registers; kNm: the N_m planes are
// written too (every row's profile is then kept until its planes are
// stored; without them a row's profile lives only while its K is formed,
// which keeps the kernel at a third of the registers).
template <int kL, bool kNm>
__global__ void __launch_bounds__(256)
k_combine(const DsInfo* __restrict__ dsv, uint32_t nds, const AccParams p, int want_khat) {
  __shared__ int32_t ti[32][33];
  __shared__ double td[32][33];
  const uint32_t b = blockIdx.x;
  uint32_t d = 0;
  while (d + 1 < nds && dsv[d + 1].tile0 <= b) ++d;
  const DsInfo D = dsv[d];
  const uint32_t n = D.n, nt = (n + 31) / 32;
  const uint32_t t = b - D.tile0;
  const uint32_t I = t / nt, J = t % nt;
  if (I > J) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const uint64_t nn = (uint64_t)n * n;
  const uint32_t M = p.M;
  // Four elements per thread: rows I*32 + ty + 8 r, column J*32 + tx.
  uint32_t Nv[kNm ? 4 : 1][kL];
  uint32_t Kv[4];
  bool up[4];
  const uint32_t col = J * 32 + tx;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint32_t row = I * 32 + ty + 8 * r;
    up[r] = row < n && col < n && row <= col;
    Kv[r] = 0;
    uint32_t* N = Nv[kNm ? r : 0];
#pragma unroll
    for (int m = 0; m < kL; ++m) N[m] = 0;
    if (up[r]) {
      uint32_t C[kL];
      const uint64_t o = (uint64_t)row * n + col;
#pragma unroll
      for (int m = 0; m < kL; ++m) C[m] = (uint32_t)m <= M ? D.C[m * nn + o] : 0u;
      Kv[r] = ie_combine<kL>(C, M, p.ie, p.h, N);
      uint32_t CM = 0;
#pragma unroll
      for (int m = 0; m < kL; ++m)
        if ((uint32_t)m == M) CM = C[m];
      if (Kv[r] != CM) atomicOr(p.status, kErrKneCM);
    }
  }
  // Plane 0 is K, planes 1..M+1 are N_0..N_M: upper write, then the
  // mirrored lower write.
  const int nplanes = 1 + ((kNm && D.Nm) ? (int)M + 1 : 0);
  for (int pl = 0; pl < nplanes; ++pl) {
    int32_t* X = pl == 0 ? D.K : D.Nm + (uint64_t)(pl - 1) * nn;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      uint32_t v = Kv[r];
      if constexpr (kNm) {
#pragma unroll
        for (int m = 0; m < kL; ++m)
          if (m == pl - 1) v = Nv[r][m];
      }
      const uint32_t row = I * 32 + ty + 8 * r;
      if (up[r]) X[(uint64_t)row * n + col] = (int32_t)v;
      ti[ty + 8 * r][tx] = (int32_t)v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // Output (J*32 + ty + 8r, I*32 + tx) mirrors source (I*32 + tx, J*32 + ty + 8r).
      const uint32_t orow = J * 32 + ty + 8 * r, ocol = I * 32 + tx;
      if (orow < n && ocol < n && ocol < orow) X[(uint64_t)orow * n + ocol] = ti[tx][ty + 8 * r];
    }
    __syncthreads();
  }
  if (want_khat && D.Khat) {
    const double rc = col < n ? D.rinv[col] : 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t row = I * 32 + ty + 8 * r;
      double v = 0.0;
      if (up[r]) {
        if (row == col)
          v = D.rinv[row] > 0.0 ? 1.0 : 0.0;
        else
          v = ((double)Kv[r] * D.rinv[row]) * rc;
        D.Khat[(uint64_t)row * n + col] = v;
      }
      td[ty + 8 * r][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t orow = J * 32 + ty + 8 * r, ocol = I * 32 + tx;
      if (orow < n && ocol < n && ocol < orow) D.Khat[(uint64_t)orow * n + ocol] = td[tx][ty + 8 * r];
    }
  }
}

// Mirror the strict lower triangle of K (and of each N_m) from the upper
// triangle, and write the normalised kernel
//   Khat(x, y) = K(x, y) / sqrt(K(x, x) K(y, y)),
// computed as (K * r_x) * r_y with r = 1 / sqrt(K(x, x)) (relative error a
// few ulp), exactly 1 on a nonzero diagonal and 0 where a diagonal is 0.
// One block per 32 x 32 output tile.
__global__ void __launch_bounds__(256)
k_finish(const DsInfo* __restrict__ dsv, uint32_t nds, uint32_t M, int want_nm,
         int want_khat) {
  __shared__ int32_t tile[32][33];
  const uint32_t b = blockIdx.x;
  uint32_t d = 0;
  while (d + 1 < nds && dsv[d + 1].tile0 <= b) ++d;
  const DsInfo D = dsv[d];
  const uint32_t n = D.n, nt = (n + 31) / 32;
  const uint32_t t = b - D.tile0;
  const uint32_t I = t / nt, J = t % nt;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const uint64_t nn = (uint64_t)n * n;
  const int nplanes = 1 + ((want_nm && D.Nm) ? (int)M + 1 : 0);
  for (int pl = 0; pl < nplanes; ++pl) {
    int32_t* X = pl == 0 ? D.K : D.Nm + (uint64_t)(pl - 1) * nn;
    if (I >= J) {
      for (int r = ty; r < 32; r += 8) {
        const uint32_t row = J * 32 + r, col = I * 32 + tx;
        if (row < n && col < n) tile[r][tx] = X[(uint64_t)row * n + col];
      }
      __syncthreads();
      for (int r = ty; r < 32; r += 8) {
        const uint32_t row = I * 32 + r, col = J * 32 + tx;
        if (row < n && col < n && row > col) X[(uint64_t)row * n + col] = tile[tx][r];
      }
    }
    if (pl == 0 && want_khat && D.Khat) {
      for (int r = ty; r < 32; r += 8) {
        const uint32_t row = I * 32 + r, col = J * 32 + tx;
        if (row >= n || col >= n) continue;
        int32_t k;
        if (I > J || (I == J && row > col))
          k = tile[tx][r];
        else if (I == J)
          k = tile[r][tx];
        else
          k = X[(uint64_t)row * n + col];
        double v;
        if (row == col)
          v = D.rinv[row] > 0.0 ? 1.0 : 0.0;
        else
          v = ((double)k * D.rinv[row]) * D.rinv[col];
        D.Khat[(uint64_t)row * n + col] = v;
      }
    }
    __syncthreads();
  }
}

// countAndUpdate exactly as Alg. 1 states it: one thread per entry
// (f, x, c_x) adds c_x * c_y into the global C_m(x, y) for every entry
// (f, y, c_y) of its feature with y >= x.
__global__ void __launch_bounds__(256)
k_pairs_global(const uint32_t* __restrict__ segtot_E, const uint32_t* __restrict__ eseq,
               const uint32_t* __restrict__ efe, uint32_t* __restrict__ Cm, uint32_t n,
               uint32_t* __restrict__ status) {
  const uint32_t E = *segtot_E;
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const uint32_t v = eseq[e];
  const uint64_t row = (uint64_t)(v >> 16) * n;
  const uint32_t c = v & 0xFFFFu, hi = efe[e];
  if (hi > E || (v >> 16) >= n) {
    atomicOr(status, kErrBadEntry);
    return;
  }
  for (uint32_t e2 = e; e2 < hi; ++e2) {
    const uint32_t v2 = eseq[e2];
    if ((v2 >> 16) < n)
      atomicAdd(&Cm[row + (v2 >> 16)], c * (v2 & 0xFFFFu));
    else
      atomicOr(status, kErrBadEntry);
  }
}

// Eq. 9 and Eq. 7 over the upper triangle of the global C_0..C_M.
__global__ void __launch_bounds__(256)
k_ie_combine(const DsInfo* __restrict__ dsv, const uint32_t* __restrict__ Cg,
             const AccParams p) {
  const DsInfo D = *dsv;
  const uint64_t nn = (uint64_t)D.n * D.n;
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < nn;
       o += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = (uint32_t)(o / D.n), y = (uint32_t)(o % D.n);
    if (y < x) continue;
    uint32_t C[kMaxLevels], N[kMaxLevels];
#pragma unroll
    for (int m = 0; m < kMaxLevels; ++m) C[m] = (uint32_t)m <= p.M ? Cg[m * nn + o] : 0u;
    const uint32_t K = ie_combine(C, p.M, p.ie, p.h, N);
    uint32_t CM = 0;
#pragma unroll
    for (int m = 0; m < kMaxLevels; ++m)
      if ((uint32_t)m == p.M) CM = C[m];
    if (K != CM) atomicOr(p.status, kErrKneCM);
    D.K[o] = (int32_t)K;
    if (D.Nm) {
#pragma unroll
      for (int m = 0; m < kMaxLevels; ++m)
        if ((uint32_t)m <= p.M) D.Nm[m * nn + o] = (int32_t)N[m];
    }
    if (y == x) D.rinv[x] = K ? 1.0 / sqrt((double)K) : 0.0;
  }
}

}  // namespace

int accum_max_threads() { return 1024; }

template <int T, int V>
static void accum_t(const AccParams& p, int blocks, size_t smem, cudaStream_t st) {
  k_accum<T, V><<<blocks, T, smem, st>>>(p);
}

template <int V>
static void accum_v(const AccParams& p, int threads, int blocks, size_t smem, cudaStream_t st) {
  if (threads == 256)
    accum_t<256, V>(p, blocks, smem, st);
  else if (threads == 1024)
    accum_t<1024, V>(p, blocks, smem, st);
  else
    accum_t<512, V>(p, blocks, smem, st);
}

void launch_accum(const AccParams& p, int threads, int variant, int blocks, size_t smem,
                  cudaStream_t st) {
  if (p.nitems == 0) return;
  if (variant == 1)
    accum_v<1>(p, threads, blocks, smem, st);
  else if (variant == 2)
    accum_v<2>(p, threads, blocks, smem, st);
  else
    accum_v<0>(p, threads, blocks, smem, st);
}

template <int T, int V>
static int accum_occ(size_t smem) {
  int nb = 0;
  cudaError_t e = cudaFuncSetAttribute(k_accum<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_accum<T, V>, T, smem);
  return e ? -1 : nb;
}

template <int V>
static int accum_occ_v(int threads, size_t smem) {
  if (threads == 256) return accum_occ<256, V>(smem);
  if (threads == 1024) return accum_occ<1024, V>(smem);
  return accum_occ<512, V>(smem);
}

int accum_blocks_per_sm(int threads, int variant, size_t smem) {
  if (variant == 1) return accum_occ_v<1>(threads, smem);
  if (variant == 2) return accum_occ_v<2>(threads, smem);
  return accum_occ_v<0>(threads, smem);
}

void launch_finish(const DsInfo* d_ds, uint32_t nds, uint32_t ntiles, uint32_t M,
                   bool want_nm, bool want_khat, cudaStream_t st) {
  if (ntiles == 0) return;
  k_finish<<<ntiles, 256, 0, st>>>(d_ds, nds, M, want_nm ? 1 : 0, want_khat ? 1 : 0);
}

void launch_diag(const DsInfo* d_ds, uint32_t nds, uint32_t nseq_total, const AccParams& coef,
                 cudaStream_t st) {
  if (nseq_total == 0) return;
  k_diag<<<(nseq_total + 255) / 256, 256, 0, st>>>(d_ds, nds, nseq_total, coef);
}

void launch_combine(const DsInfo* d_ds, uint32_t nds, uint32_t ntiles, const AccParams& coef,
                    bool want_nm, bool want_khat, cudaStream_t st) {
  if (ntiles == 0) return;
  const int kh = want_khat ? 1 : 0;
  // want_nm asks for the planes; a dataset without an N_m buffer writes none.
  if (coef.M + 1 <= 8) {
    if (want_nm)
      k_combine<8, true><<<ntiles, 256, 0, st>>>(d_ds, nds, coef, kh);
    else
      k_combine<8, false><<<ntiles, 256, 0, st>>>(d_ds, nds, coef, kh);
  } else {
    if (want_nm)
      k_combine<kMaxLevels, true><<<ntiles, 256, 0, st>>>(d_ds, nds, coef, kh);
    else
      k_combine<kMaxLevels, false><<<ntiles, 256, 0, st>>>(d_ds, nds, coef, kh);
  }
}

void launch_pairs_global(const uint32_t* segtot_E, const uint32_t* eseq,
                         const uint32_t* efe, uint32_t G, uint32_t* Cm, uint32_t n,
                         uint32_t* status, cudaStream_t st) {
  if (G == 0) return;
  k_pairs_global<<<(G + 255) / 256, 256, 0, st>>>(segtot_E, eseq, efe, Cm, n, status);
}

void launch_ie_combine(const DsInfo* d_ds, const uint32_t* C, uint32_t n,
                       const AccParams& coef, cudaStream_t st) {
  const uint64_t nn = (uint64_t)n * n;
  if (nn == 0) return;
  uint64_t blocks = (nn + 255) / 256;
  if (blocks > 65535ull * 16) blocks = 65535ull * 16;
  k_ie_combine<<<(unsigned)blocks, 256, 0, st>>>(d_ds, C, coef);
}

}  // namespace gk
