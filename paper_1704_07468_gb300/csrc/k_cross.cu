// Cross kernel K(test, train) against a resident training set.
//
// The paper classifies with one kernel over training and test sequences
// together (Section 3.1); the test-rows x train-columns block of that kernel
// is K(test, train), and each test diagonal K(t, t) depends on t alone.
// Here the training side is indexed once ("fit"): for every mask, its
// features (distinct (g-m)-mers) in key order with the range of their
// entries, and the training diagonal.  A test batch is sorted and counted
// per mask like a dataset of its own; each test entry (f, t, c_t) is joined
// to the training feature with the same key by binary search, and the
// accumulation adds c_t * c_y over that feature's training entries
// (Section 2.2, steps 2-5), for every training column.  Eq. 9 and Eq. 7
// then give N_m and K, and K is normalised with both diagonals.
#include <cstdint>

#include "common.cuh"
#include "launch.h"

namespace gk {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kLong = 32;

__device__ __forceinline__ uint32_t ie_kernel(const uint32_t* C, uint32_t M,
                                              const uint32_t (*ie)[kMaxLevels],
                                              const uint32_t* h, uint32_t* N) {
  uint32_t K = 0;
#pragma unroll
  for (int m = 0; m < kMaxLevels; ++m) {
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

// Training index of one sorted and counted chunk: per feature its key and
// first entry, the entries themselves, and C_m(y, y) += c^2 per entry.
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads)
k_train_index(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
              const uint32_t* __restrict__ segtot, const KeyT* __restrict__ keys,
              const uint32_t* __restrict__ estart, const uint32_t* __restrict__ fstart,
              const uint32_t* __restrict__ eseq, const uint32_t* __restrict__ mask_level,
              TrainIndex tr) {
  const uint32_t t = blockIdx.x;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t lt = t - sd.tile0;
  const uint32_t E = segtot[2 * s], F = segtot[2 * s + 1];
  const uint64_t tb = sd.base + s;
  const uint64_t tp = (uint64_t)sd.mask * tr.stride;
  const uint32_t lvl = mask_level[sd.mask];
  const uint64_t beg = (uint64_t)lt * kTile;
  for (uint32_t q = threadIdx.x; q < kTile; q += blockDim.x) {
    const uint64_t i = beg + q;
    if (i < F) {
      const uint32_t fe = fstart[tb + i];
      tr.ufirst[tp + i] = fe;
      tr.ukey[tp + i] = (uint64_t)keys[sd.base + estart[tb + fe]];
      if (i + 1 == F) {
        tr.ufirst[tp + F] = E;
        tr.nfeat[sd.mask] = F;
      }
    }
    if (i < E) {
      const uint32_t v = eseq[sd.pool + i];
      tr.eseq[tp + i] = v;
      const uint32_t c = v & 0xFFFFu;
      atomicAdd(&tr.diagC[(uint64_t)lvl * tr.n + (v >> 16)], c * c);
    }
  }
  if (F == 0 && lt == 0 && threadIdx.x == 0) {
    tr.ufirst[tp] = 0;
    tr.nfeat[sd.mask] = 0;
  }
}

// Test entries of one chunk: entry word, count^2 into the test diagonal,
// and the entry range [a, b) of the training feature with the same key.
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads)
k_cross_final(const SegDesc* __restrict__ segs, const uint32_t* __restrict__ tile_seg,
              const uint32_t* __restrict__ segtot, const KeyT* __restrict__ keys,
              const uint32_t* __restrict__ estart, const uint32_t* __restrict__ etseq,
              const uint32_t* __restrict__ mask_level, TrainIndex tr, CrossOut xo) {
  const uint32_t t = blockIdx.x;
  const uint32_t s = tile_seg[t];
  const SegDesc sd = segs[s];
  const uint32_t lt = t - sd.tile0;
  const uint32_t E = segtot[2 * s];
  const uint64_t tb = sd.base + s;
  const uint64_t tp = (uint64_t)sd.mask * tr.stride;
  const uint32_t nf = tr.nfeat[sd.mask];
  const uint32_t lvl = mask_level[sd.mask];
  const uint64_t beg = (uint64_t)lt * kTile;
  for (uint32_t q = threadIdx.x; q < kTile; q += blockDim.x) {
    const uint64_t e = beg + q;
    if (e >= E) break;
    const uint32_t st = estart[tb + e];
    const uint32_t c = estart[tb + e + 1] - st;
    const uint32_t seq = etseq[tb + e];
    xo.eseq[sd.pool + e] = (seq << 16) | c;
    atomicAdd(&xo.Cd[(uint64_t)lvl * xo.nt + seq], c * c);
    const uint64_t key = (uint64_t)keys[sd.base + st];
    uint32_t lo = 0, hi = nf;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (tr.ukey[tp + mid] < key)
        lo = mid + 1;
      else
        hi = mid;
    }
    uint32_t a = 0, b = 0;
    if (lo < nf && tr.ukey[tp + lo] == key) {
      a = tr.ufirst[tp + lo];
      b = tr.ufirst[tp + lo + 1];
    }
    xo.ea[sd.pool + e] = a;
    xo.eb[sd.pool + e] = b;
  }
}

// First entry in [lo, hi) whose sequence is >= seq.
__device__ __forceinline__ uint32_t lower_bound_seq(const uint32_t* __restrict__ es, uint32_t lo,
                                                    uint32_t hi, uint32_t seq) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((es[mid] >> 16) < seq)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// One row t of C_m(t, .) over training columns [c0, c1) for a group of a
// level's masks; added to the global Cx with reductions.
template <int kThreads>
__global__ void __launch_bounds__(kThreads)
k_cross_accum(const CrossParams p) {
  extern __shared__ uint32_t acc[];   // ncols + 1 (trash slot)
  __shared__ uint32_t s_item;
  constexpr int kWarps = kThreads / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(p.counter, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= p.nitems) return;
    const uint32_t* I = p.items + (uint64_t)it * kItemWords;
    const uint32_t lvl = I[1], mfirst = I[2], mcount = I[3];
    const uint32_t x = I[4], c0 = I[5], c1 = I[6];
    const uint32_t width = c1 - c0;
    for (uint32_t i = threadIdx.x; i <= width; i += kThreads) acc[i] = 0;
    __syncthreads();
    const uint32_t wbeg = p.woff[x], wend = p.woff[x + 1];
    const bool lo_cut = c0 > 0, hi_cut = c1 < p.tr.n;
    const uint32_t nch = (wend - wbeg + 31) / 32;
    for (uint32_t ch = w; ch < mcount * nch; ch += kWarps) {
      const uint32_t mu = mfirst + ch / nch;
      const uint32_t wi = wbeg + (ch % nch) * 32 + lane;
      const uint64_t pool = (uint64_t)mu * p.gt;
      const uint32_t* __restrict__ tes = p.tr.eseq + (uint64_t)mu * p.tr.stride;
      uint32_t e = wi < wend ? p.ewin[pool + wi] : kNone;
      uint32_t lo = 0, cnt = 0, c = 0;
      if (e != kNone) {
        c = p.xo.eseq[pool + e] & 0xFFFFu;
        lo = p.xo.ea[pool + e];
        uint32_t hi = p.xo.eb[pool + e];
        if (hi > p.tr.stride || lo > hi) {
          atomicOr(p.status, kErrBadEntry);
          hi = lo;
        }
        if (lo_cut) lo = lower_bound_seq(tes, lo, hi, c0);
        if (hi_cut) hi = lower_bound_seq(tes, lo, hi, c1);
        cnt = hi - lo;
      }
      uint32_t longm = __ballot_sync(kFull, cnt >= kLong);
      while (longm) {
        const int L = __ffs(longm) - 1;
        longm &= longm - 1;
        const uint32_t lL = __shfl_sync(kFull, lo, L);
        const uint32_t nL = __shfl_sync(kFull, cnt, L);
        const uint32_t cL = __shfl_sync(kFull, c, L);
        const uint32_t* __restrict__ src = tes + lL;
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
      // Short ranges: up to four pairs per lane directly, the rest by a
      // warp-wide expansion.
      {
        const uint32_t s4 = min(cnt, 4u);
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (uint32_t)u < s4 ? tes[lo + u] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((uint32_t)u < s4) atomicAdd(&acc[min((v[u] >> 16) - c0, width)], c * (v[u] & 0xFFFFu));
        lo += s4;
        cnt -= s4;
      }
      if (__any_sync(kFull, cnt != 0)) {
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const uint32_t excl = incl - cnt;
        for (uint32_t p0 = 0; p0 < total; p0 += 32) {
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
            const uint32_t v = tes[lo_o + (pp - ex_o)];
            atomicAdd(&acc[min((v >> 16) - c0, width)], c_o * (v & 0xFFFFu));
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && acc[width] != 0) atomicOr(p.status, kErrBadEntry);
    uint32_t* __restrict__ crow = p.xo.Cx + ((uint64_t)lvl * p.xo.nt + x) * p.tr.n + c0;
    for (uint32_t i = threadIdx.x; i < width; i += kThreads) {
      const uint32_t v = acc[i];
      if (v) atomicAdd(&crow[i], v);
    }
  }
}

// K(x, x) and 1/sqrt(K(x, x)) from per-level diagonals C[m * n + x].
__global__ void __launch_bounds__(256)
k_vec_diag(const uint32_t* __restrict__ Cd, uint32_t n, const CrossParams p, double* __restrict__ rinv) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  uint32_t C[kMaxLevels], N[kMaxLevels];
#pragma unroll
  for (int m = 0; m < kMaxLevels; ++m) C[m] = (uint32_t)m <= p.M ? Cd[(uint64_t)m * n + x] : 0u;
  const uint32_t K = ie_kernel(C, p.M, p.ie, p.h, N);
  rinv[x] = K ? 1.0 / sqrt((double)K) : 0.0;
}

// K(t, y) and Khat(t, y) = (K * r_t) * r_y for every test row and training
// column, with the identity K == C_M checked.
__global__ void __launch_bounds__(256)
k_cross_combine(const CrossParams p, int32_t* __restrict__ K, double* __restrict__ Khat) {
  const uint64_t total = (uint64_t)p.xo.nt * p.tr.n;
  const uint64_t plane = total;
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < total;
       o += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(o / p.tr.n), y = (uint32_t)(o % p.tr.n);
    uint32_t C[kMaxLevels], N[kMaxLevels];
#pragma unroll
    for (int m = 0; m < kMaxLevels; ++m) C[m] = (uint32_t)m <= p.M ? p.xo.Cx[m * plane + o] : 0u;
    const uint32_t k = ie_kernel(C, p.M, p.ie, p.h, N);
    uint32_t CM = 0;
#pragma unroll
    for (int m = 0; m < kMaxLevels; ++m)
      if ((uint32_t)m == p.M) CM = C[m];
    if (k != CM) atomicOr(p.status, kErrKneCM);
    if (K) K[o] = (int32_t)k;
    if (Khat) Khat[o] = ((double)k * p.xo.rinv[t]) * p.tr.rinv[y];
  }
}

// SVM decision values (Eq. 1): f(t) = sum_y coef[y] k(t, y) + bias with
// coef[y] = alpha_y * label_y supplied by the caller and k = Khat (kind 0,
// computed exactly as k_cross_combine writes it) or K (kind 1).  One block
// per test row and a fixed-order reduction, so a row's value does not
// depend on the batch it ran in.
__global__ void __launch_bounds__(256)
k_svm_decision(const CrossParams p, const double* __restrict__ coef, double bias, int kind,
               double* __restrict__ f) {
  __shared__ double red[256];
  const uint32_t t = blockIdx.x;
  const uint64_t plane = (uint64_t)p.xo.nt * p.tr.n;
  double acc = 0.0;
  for (uint32_t y = threadIdx.x; y < p.tr.n; y += 256) {
    const uint64_t o = (uint64_t)t * p.tr.n + y;
    uint32_t C[kMaxLevels], N[kMaxLevels];
#pragma unroll
    for (int m = 0; m < kMaxLevels; ++m) C[m] = (uint32_t)m <= p.M ? p.xo.Cx[m * plane + o] : 0u;
    const uint32_t k = ie_kernel(C, p.M, p.ie, p.h, N);
    const double v = kind ? (double)k : ((double)k * p.xo.rinv[t]) * p.tr.rinv[y];
    acc += coef[y] * v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (uint32_t s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) f[t] = red[0] + bias;
}

// ----------------------------------------------------- merging indexes --
//
// Adding sequences to a fitted set (Section 3.2, Fig. 5(c)): the index b of
// the new sequences (their ids offset by seq_off) is merged into the
// resident index a.  Per mask the merged features are the union of both
// key lists in key order, and each feature's entries are a's followed by
// b's (the new sequences have the larger ids), which is the index a fit of
// the union builds.  With rb(j) = features of a with a smaller key than
// b's feature j, ra(i) the same for a's feature i in b, and cb(j) = b's
// features before j whose key a also holds:
//   merged position of a's feature i      i + ra(i) - cb(ra(i))
//   merged position of b's feature j      rb(j) + j - cb(j)   (key not in a)
//   first entry of a's feature i          a.first(i) + b.first(ra(i))
//   first entry of b's feature j          a.first(rb(j)) + b.first(j)
// and an entry of a's feature i moves by b.first(ra(i)).

__device__ __forceinline__ uint32_t lower_bound_key(const uint64_t* __restrict__ k, uint32_t n, uint64_t key) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (k[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Grid (blocks, masks): rb(j), and a flag "a holds the key" in cb (scanned
// in place by k_merge_scan).
__global__ void __launch_bounds__(256)
k_merge_rank(const TrainIndex a, const TrainIndex b, uint32_t* __restrict__ rb, uint32_t* __restrict__ cb) {
  const uint32_t mu = blockIdx.y;
  const uint32_t Fa = a.nfeat[mu], Fb = b.nfeat[mu];
  const uint64_t* __restrict__ ka = a.ukey + (uint64_t)mu * a.stride;
  const uint64_t ob = (uint64_t)mu * b.stride;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < Fb; j += gridDim.x * blockDim.x) {
    const uint64_t k = b.ukey[ob + j];
    const uint32_t r = lower_bound_key(ka, Fa, k);
    rb[ob + j] = r;
    cb[ob + j] = (r < Fa && ka[r] == k) ? 1u : 0u;
  }
}

// One block per mask: exclusive scan of the flags (their total at cb(Fb)),
// then the merged feature count and the merged end-of-entries sentinel.
__global__ void __launch_bounds__(1024)
k_merge_scan(const TrainIndex a, const TrainIndex b, TrainIndex m, uint32_t* __restrict__ cb) {
  __shared__ uint32_t sw[33];
  const uint32_t mu = blockIdx.x;
  const uint32_t Fb = b.nfeat[mu];
  uint32_t* __restrict__ c = cb + (uint64_t)mu * b.stride;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < Fb; base += blockDim.x) {
    const uint32_t j = base + threadIdx.x;
    const uint32_t v = j < Fb ? c[j] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) sw[w] = incl;
    __syncthreads();
    if (w == 0) {
      const uint32_t x = lane < nw ? sw[lane] : 0u;
      uint32_t xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, xi, o);
        if (lane >= (uint32_t)o) xi += t;
      }
      if (lane < nw) sw[lane] = xi - x;
      if (lane == 31) sw[32] = xi;
    }
    __syncthreads();
    if (j < Fb) c[j] = carry + sw[w] + incl - v;
    carry += sw[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c[Fb] = carry;
    const uint32_t Fa = a.nfeat[mu];
    const uint32_t Fm = Fa + Fb - carry;
    m.nfeat[mu] = Fm;
    m.ufirst[(uint64_t)mu * m.stride + Fm] =
        a.ufirst[(uint64_t)mu * a.stride + Fa] + b.ufirst[(uint64_t)mu * b.stride + Fb];
  }
}

// Grid (blocks, masks), a warp per 32 consecutive features of a: their
// merged records, their entries (the warp copies the 32 features' entry
// span with consecutive lanes on consecutive entries, each entry moved by
// its feature's shift, found by a search over the lanes), then b's entries
// of the features both indexes hold.
__global__ void __launch_bounds__(256)
k_merge_old(const TrainIndex a, const TrainIndex b, TrainIndex m, const uint32_t* __restrict__ cb,
            uint32_t seq_off) {
  const uint32_t mu = blockIdx.y;
  const uint32_t Fa = a.nfeat[mu], Fb = b.nfeat[mu];
  const uint64_t oa = (uint64_t)mu * a.stride, ob = (uint64_t)mu * b.stride, om = (uint64_t)mu * m.stride;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; i0 < Fa; i0 += nwarps * 32) {
    const uint32_t i = i0 + lane;
    const uint32_t nv = min(32u, Fa - i0);
    uint32_t f0 = 0, f1 = 0, sh = 0, rn = 0;
    uint64_t k = 0;
    if (lane < nv) {
      k = a.ukey[oa + i];
      f0 = a.ufirst[oa + i];
      f1 = a.ufirst[oa + i + 1];
      rn = lower_bound_key(b.ukey + ob, Fb, k);
      sh = b.ufirst[ob + rn];
      const uint32_t pm = i + rn - cb[ob + rn];
      m.ukey[om + pm] = k;
      m.ufirst[om + pm] = f0 + sh;
    }
    const uint32_t s0 = __shfl_sync(kFull, f0, 0), s1 = __shfl_sync(kFull, f1, nv - 1);
    for (uint32_t e0 = s0; e0 < s1; e0 += 32) {
      const uint32_t e = e0 + lane;
      uint32_t L = 0;  // last valid lane whose first entry is <= e
#pragma unroll
      for (uint32_t step = 16; step >= 1; step >>= 1) {
        const uint32_t t = __shfl_sync(kFull, f0, L + step);
        if (L + step < nv && t <= e) L += step;
      }
      const uint32_t s = __shfl_sync(kFull, sh, L);
      if (e < s1) m.eseq[om + e + s] = a.eseq[oa + e];
    }
    if (lane < nv && rn < Fb && b.ukey[ob + rn] == k) {
      const uint32_t q0 = b.ufirst[ob + rn], q1 = b.ufirst[ob + rn + 1];
      for (uint32_t q = q0; q < q1; ++q) m.eseq[om + f1 + sh + (q - q0)] = b.eseq[ob + q] + (seq_off << 16);
    }
  }
}

// Grid (blocks, masks): b's features whose key a does not hold.
__global__ void __launch_bounds__(256)
k_merge_new(const TrainIndex a, const TrainIndex b, TrainIndex m, const uint32_t* __restrict__ rb,
            const uint32_t* __restrict__ cb, uint32_t seq_off) {
  const uint32_t mu = blockIdx.y;
  const uint32_t Fa = a.nfeat[mu], Fb = b.nfeat[mu];
  const uint64_t oa = (uint64_t)mu * a.stride, ob = (uint64_t)mu * b.stride, om = (uint64_t)mu * m.stride;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < Fb; j += gridDim.x * blockDim.x) {
    const uint32_t ro = rb[ob + j];
    const uint64_t k = b.ukey[ob + j];
    if (ro < Fa && a.ukey[oa + ro] == k) continue;  // placed with a's feature
    const uint32_t pm = ro + j - cb[ob + j];
    const uint32_t q0 = b.ufirst[ob + j], q1 = b.ufirst[ob + j + 1];
    const uint32_t ef = a.ufirst[oa + ro] + q0;
    m.ukey[om + pm] = k;
    m.ufirst[om + pm] = ef;
    for (uint32_t q = q0; q < q1; ++q) m.eseq[om + ef + (q - q0)] = b.eseq[ob + q] + (seq_off << 16);
  }
}

}  // namespace

void launch_svm_decision(const CrossParams& p, const double* coef, double bias, int kind, double* f,
                         cudaStream_t st) {
  if (p.xo.nt == 0) return;
  k_svm_decision<<<p.xo.nt, 256, 0, st>>>(p, coef, bias, kind, f);
}

void launch_train_index(bool wide, const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                        const uint32_t* segtot, const void* keys, const uint32_t* estart,
                        const uint32_t* fstart, const uint32_t* eseq, const uint32_t* mask_level,
                        const TrainIndex& tr, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    k_train_index<uint64_t><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, segtot, (const uint64_t*)keys,
                                                             estart, fstart, eseq, mask_level, tr);
  else
    k_train_index<uint32_t><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, segtot, (const uint32_t*)keys,
                                                             estart, fstart, eseq, mask_level, tr);
}

void launch_cross_final(bool wide, const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                        const uint32_t* segtot, const void* keys, const uint32_t* estart,
                        const uint32_t* etseq, const uint32_t* mask_level, const TrainIndex& tr,
                        const CrossOut& xo, cudaStream_t st) {
  if (ntiles == 0) return;
  if (wide)
    k_cross_final<uint64_t><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, segtot, (const uint64_t*)keys,
                                                             estart, etseq, mask_level, tr, xo);
  else
    k_cross_final<uint32_t><<<ntiles, kSortThreads, 0, st>>>(segs, tile_seg, segtot, (const uint32_t*)keys,
                                                             estart, etseq, mask_level, tr, xo);
}

int cross_accum_blocks_per_sm(size_t smem) {
  int nb = 0;
  cudaError_t e = cudaFuncSetAttribute(k_cross_accum<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cross_accum<512>, 512, smem);
  return e ? -1 : nb;
}

void launch_cross_accum(const CrossParams& p, int blocks, size_t smem, cudaStream_t st) {
  if (p.nitems == 0) return;
  k_cross_accum<512><<<blocks, 512, smem, st>>>(p);
}

void launch_vec_diag(const uint32_t* Cd, uint32_t n, const CrossParams& p, double* rinv, cudaStream_t st) {
  if (n == 0) return;
  k_vec_diag<<<(n + 255) / 256, 256, 0, st>>>(Cd, n, p, rinv);
}

void launch_cross_combine(const CrossParams& p, int32_t* K, double* Khat, cudaStream_t st) {
  const uint64_t total = (uint64_t)p.xo.nt * p.tr.n;
  if (total == 0) return;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 152ull * 64) blocks = 152ull * 64;
  k_cross_combine<<<(unsigned)blocks, 256, 0, st>>>(p, K, Khat);
}

void launch_index_merge(const TrainIndex& a, const TrainIndex& b, const TrainIndex& m, uint32_t nmasks,
                        uint32_t* rb, uint32_t* cb, uint32_t seq_off, cudaStream_t st) {
  if (nmasks == 0) return;
  const dim3 grid(32, nmasks);
  k_merge_rank<<<grid, 256, 0, st>>>(a, b, rb, cb);
  k_merge_scan<<<nmasks, 1024, 0, st>>>(a, b, m, cb);
  k_merge_old<<<grid, 256, 0, st>>>(a, b, m, cb, seq_off);
  k_merge_new<<<grid, 256, 0, st>>>(a, b, m, rb, cb, seq_off);
}

}  // namespace gk
