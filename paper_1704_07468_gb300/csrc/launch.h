// Host-side launch wrappers of the engine's kernels (one definition per .cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gk {

// Per-dataset description for the g-mer packing kernel.
struct DsPack {
  const uint8_t* codes;   // device, symbols of all sequences concatenated
  const int64_t* coff;    // device, n + 1 code offsets
  const uint32_t* woff;   // device, n + 1 window offsets
  uint64_t win0;          // first global window
  uint32_t n;
  uint32_t seq0;          // first global sequence
};

// k_prep.cu -------------------------------------------------------------
int prep_init();  // one-time kernel attributes; returns a cudaError_t
void launch_pack(const DsPack* d_ds, uint32_t nds, uint32_t nseq_total,
                 int g, int bits, int sigma, uint64_t* fullkey,
                 uint32_t* wid, uint32_t* status, cudaStream_t st);

// One LSD radix-sort pass over every segment of a chunk.  For the first
// pass the keys are cut out of the full g-mer keys (`fullkey`) into `kin`
// (which must not alias `kout`) and the payload is the window id read from
// `vin` (the packing kernel's output, indexed by global window); later
// passes read kin/vin.  dtot: nsegs << rbits words of scratch (each
// segment's digit totals, then the digits' starts).
void launch_sort_pass(bool wide, bool first, const SegDesc* segs,
                      uint32_t nsegs, const uint32_t* tile_seg,
                      uint32_t ntiles, const MaskDesc* masks,
                      const uint64_t* fullkey, void* kin,
                      const uint32_t* vin, void* kout, uint32_t* vout,
                      uint32_t* hist, uint32_t* dtot, int shift, int rbits, cudaStream_t st);

// Onesweep form of the same sort (digits of at most 8 bits): the digit
// counts of every pass of a chunk in one read of the keys, then one scatter
// per pass with a decoupled look-back.
constexpr int kOsMaxPasses = 8;
constexpr int kOsRadix = 256;
struct OsPasses {
  int np;
  int shift[kOsMaxPasses];
  int bits[kOsMaxPasses];
};
// Cuts the masked keys into kx and adds every pass's digit counts of each
// segment into dcount[(segment * np + pass) * kOsRadix + digit] (zeroed by
// the caller), then turns them into each digit's start in its segment.
void launch_os_hist(bool wide, const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg,
                    uint32_t ntiles, const MaskDesc* masks, const uint64_t* fullkey, void* kx,
                    uint32_t* dcount, const OsPasses& ps, cudaStream_t st);
// Pass q: tiles taken in order from *ctr (zero before the launch); st holds
// kOsRadix status words per tile, whose epochs must differ from `epoch`
// (1..65535) unless written by this pass.
void launch_os_scatter(bool wide, bool first, const SegDesc* segs, const uint32_t* tile_seg,
                       uint32_t ntiles, const void* kin, const uint32_t* vin, void* kout,
                       uint32_t* vout, const uint32_t* dbase, int np, int q, int shift, int rbits,
                       uint64_t* st, uint32_t* ctr, uint32_t epoch, uint32_t* status, cudaStream_t stm);

// Run-length pass over sorted segments: entries (feature, sequence, count)
// and features (runs of equal keys).  Writes, per segment, ewin / eseq /
// efe into the pools.
void launch_rle(bool wide, const SegDesc* segs, uint32_t nsegs,
                const uint32_t* tile_seg, uint32_t ntiles, const void* keys,
                const uint32_t* vals, const DsPack* dsp,
                uint32_t* tcnt, uint32_t* segtot, uint32_t* estart,
                uint32_t* etseq, uint32_t* efid, uint32_t* fstart,
                uint32_t* ewin, uint32_t* eseq, uint32_t* efe,
                cudaStream_t st);

// k_accum.cu ------------------------------------------------------------
struct AccParams {
  const DsInfo* ds;
  const uint32_t* items;      // kItemWords x u32 per item, see gakco.cu
  uint32_t nitems;
  uint32_t* counter;
  uint32_t M;
  uint64_t gtot;
  const uint32_t* ewin;
  const uint32_t* eseq;
  const uint32_t* efe;
  uint32_t ncols;             // columns held in shared memory
  uint32_t* status;
  unsigned long long* work;   // [0] pair updates, [1] entries visited, [2] windows visited
  uint32_t h[kMaxLevels];
  uint32_t ie[kMaxLevels][kMaxLevels];
};

// Accumulation work item: dataset, level, first mask, mask count, row,
// first column, end column.
constexpr int kItemWords = 8;

int accum_max_threads();
// variant: how a warp walks entry ranges shorter than a warp (0, 1 or 2;
// see k_accum.cu); results are identical.
void launch_accum(const AccParams& p, int threads, int variant, int blocks,
                  size_t smem, cudaStream_t st);
int accum_blocks_per_sm(int threads, int variant, size_t smem);

void launch_finish(const DsInfo* d_ds, uint32_t nds, uint32_t ntiles,
                   uint32_t M, bool want_nm, bool want_khat, cudaStream_t st);

// Batched engine tail: K(x, x) and 1/sqrt(K(x, x)) from the diagonal of
// C_0..C_M, then Eq. 9 / Eq. 7 over the upper triangle of C with the
// mirrored K, N_m and Khat written in one pass.
void launch_diag(const DsInfo* d_ds, uint32_t nds, uint32_t nseq_total,
                 const AccParams& coef, cudaStream_t st);
void launch_combine(const DsInfo* d_ds, uint32_t nds, uint32_t ntiles,
                    const AccParams& coef, bool want_nm, bool want_khat,
                    cudaStream_t st);

// Run-length pass split in two: count/scan/emit, and the final entry
// packing of the Gram engine (launch_rle = both).
void launch_rle_head(bool wide, const SegDesc* segs, uint32_t nsegs,
                     const uint32_t* tile_seg, uint32_t ntiles, const void* keys,
                     const uint32_t* vals, const DsPack* dsp,
                     uint32_t* tcnt, uint32_t* segtot, uint32_t* estart,
                     uint32_t* etseq, uint32_t* efid, uint32_t* fstart,
                     uint32_t* ewin, cudaStream_t st);
// Gram engine: count/scan, then ewin, eseq and efe written directly, and
// the tile-end fix-up; trec holds kRecWords words per tile.  The chunk's
// entries are added to *ecount.  items: elements per thread of the count
// and emit kernels (16: 256-thread blocks; 8: 512-thread blocks).
void launch_rle_gram(bool wide, const SegDesc* segs, uint32_t nsegs, const uint32_t* tile_seg,
                     uint32_t ntiles, const void* keys, const uint32_t* vals, const DsPack* dsp,
                     uint32_t* tcnt, uint32_t* segtot, uint32_t* trec, uint32_t* ewin,
                     uint32_t* eseq, uint32_t* efe, unsigned long long* ecount, int items,
                     cudaStream_t st);
void launch_rle_final(const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                      const uint32_t* segtot, const uint32_t* estart,
                      const uint32_t* etseq, const uint32_t* efid,
                      const uint32_t* fstart, uint32_t* eseq, uint32_t* efe,
                      cudaStream_t st);

// k_cross.cu ------------------------------------------------------------
// Resident index of a training set: per mask (stride entries each) the
// features' keys in ascending order, their first entries (+ one past the
// last), and the entries; the per-level diagonal and 1/sqrt(K(y, y)).
struct TrainIndex {
  uint64_t* ukey;
  uint32_t* ufirst;
  uint32_t* eseq;
  uint32_t* nfeat;      // features per mask
  uint32_t* diagC;      // (M+1) x n: C_m(y, y)
  double* rinv;         // n
  uint64_t stride;      // windows of the training set + 1
  uint32_t n;
  uint32_t pad;
};

// Per test batch: entries per mask (stride = test windows), their joined
// training ranges, the test diagonal and the cross accumulators.
struct CrossOut {
  uint32_t* eseq;
  uint32_t* ea;
  uint32_t* eb;
  uint32_t* Cd;         // (M+1) x nt
  uint32_t* Cx;         // (M+1) x nt x n_train
  double* rinv;         // nt
  uint32_t nt;
  uint32_t pad;
};

struct CrossParams {
  TrainIndex tr;
  CrossOut xo;
  const uint32_t* items;  // kItemWords per item (dataset word unused)
  uint32_t nitems;
  uint32_t* counter;
  const uint32_t* woff;   // nt + 1 test window offsets
  const uint32_t* ewin;   // masks x gt
  uint64_t gt;            // test windows
  uint32_t M;
  uint32_t* status;
  uint32_t h[kMaxLevels];
  uint32_t ie[kMaxLevels][kMaxLevels];
};

void launch_train_index(bool wide, const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                        const uint32_t* segtot, const void* keys, const uint32_t* estart,
                        const uint32_t* fstart, const uint32_t* eseq, const uint32_t* mask_level,
                        const TrainIndex& tr, cudaStream_t st);
void launch_cross_final(bool wide, const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                        const uint32_t* segtot, const void* keys, const uint32_t* estart,
                        const uint32_t* etseq, const uint32_t* mask_level, const TrainIndex& tr,
                        const CrossOut& xo, cudaStream_t st);
int cross_accum_blocks_per_sm(size_t smem);
void launch_cross_accum(const CrossParams& p, int blocks, size_t smem, cudaStream_t st);
// Merges training index b (its sequences numbered from seq_off on) into
// index a, writing index m (stride >= a's + b's windows + 1); rb and cb hold
// nmasks x b.stride words of scratch.  The four launches: ranks of b's keys
// in a, a scan of the shared-key flags (also m's feature counts and
// sentinels), a's features with their entries (and b's entries of shared
// keys), then b's other features.
void launch_index_merge(const TrainIndex& a, const TrainIndex& b, const TrainIndex& m, uint32_t nmasks,
                        uint32_t* rb, uint32_t* cb, uint32_t seq_off, cudaStream_t st);
void launch_vec_diag(const uint32_t* Cd, uint32_t n, const CrossParams& p, double* rinv,
                     cudaStream_t st);
void launch_cross_combine(const CrossParams& p, int32_t* K, double* Khat, cudaStream_t st);
// SVM decision values f[t] = sum_y coef[y] k(t, y) + bias (Eq. 1); k = Khat
// (kind 0) or K (kind 1); f holds nt values.
void launch_svm_decision(const CrossParams& p, const double* coef, double bias, int kind, double* f,
                         cudaStream_t st);

// k_dense.cu ------------------------------------------------------------
// One dense problem: the count matrix A of one dataset over a run of masks
// of one level; row x = sequence x (rows padded to a multiple of 128, the
// padding all zero), column mu * 2^key_bits + key = (mask mfirst + mu,
// masked key), entry e4m3(min(count, 16)).  C_m += A A^T runs on the
// tensor cores; counts above 16 go to the overflow list and are corrected
// exactly by the fix kernel.
struct DenseProb {
  uint8_t* A;           // e4m3 bytes, n_pad x ld, row-major
  uint32_t* C;          // n x n cumulative profile C_m of the dataset
  uint32_t* maxc;       // largest entry of A as an integer, shared by the problems of one
                        // (dataset, level) (written by the scatter kernel)
  const void* tmap;     // TMA descriptor of A (kDenseTmapBytes, 64-byte aligned)
  uint64_t ld;          // columns of A, a multiple of 128
  uint32_t n, n_pad;    // sequences; rows of A
  uint32_t ds;          // dataset (DsPack index)
  uint32_t mfirst, mcount;
  uint32_t key_bits;    // (g - m) * b
  uint32_t row0;        // first row of the problem in its wave's scatter grid
  uint32_t wmasks;      // windows of the longest sequence x masks of the (dataset, level):
                        // a row of A sums to at most this over a macro tile (0 = unknown)
  uint32_t sole;        // 1: a macro tile of this problem is the only writer of its C entries
                        // until the GEMM ends (its run covers every problem of the level)
  uint32_t pad;
};

// A count above 16: problem (plan-wide index), row, column, count.
struct DenseOvf {
  uint32_t prob, x, col, count;
};

constexpr int kDenseScatterCols = 32768;  // columns per scatter block
constexpr int kDenseTmapBytes = 128;

int dense_init();  // one-time kernel attributes; returns a cudaError_t
// Host: the TMA descriptor of a byte matrix of `rows` x `ld` (box 128 x 128,
// 128-byte swizzle).  Returns 0 on success.
int dense_encode_tmap(void* out, void* A, uint64_t ld, uint64_t rows);
// d_probs: the wave's problems (row0 relative to the wave), p0 the plan
// index of the first; overflow entries go to ovf[*ovf_n++] while below
// ovf_cap.
// full_bits: bits of the packed g-mer keys (g * bits per symbol).
void launch_dense_scatter(const DenseProb* d_probs, uint32_t nprobs, uint32_t p0, uint32_t rows,
                          const DsPack* dsp, const MaskDesc* masks, const uint64_t* fullkey,
                          uint32_t full_bits, uint32_t* ovf_n, DenseOvf* ovf, uint32_t ovf_cap,
                          cudaStream_t st);
// Macro tiles of kDenseTileWords words: first problem, problem count (the
// consecutive problems of one dataset and level, whose columns the tile
// sweeps), I2, J2 (256-row and 256-column blocks, I2 <= J2), and the range
// [s0, s1) of the run's 128-column stages the tile sweeps (0, ~0 = all; a
// tile of the last, partial wave of CTAs may be cut into K-parts).
constexpr int kDenseTileWords = 6;
// Largest partial sum of one exact accumulation round: f32 holds every
// integer up to 2^24.
constexpr uint32_t kDenseExactSum = (1u << 24) - 1;
// sum_cap: bound on a round's partial sums (0 or above kDenseExactSum:
// kDenseExactSum); wait_cycles: limit of each wait between the roles
// (<= 0: about 2 s).
void launch_dense_gemm(const DenseProb* d_probs, const uint32_t* d_tiles, uint32_t ntiles, int nsm,
                       uint32_t sum_cap, long long wait_cycles, uint32_t* status, cudaStream_t st);
// d_probs: every problem of the plan.  Raises kErrDenseOverflow when the
// list overflowed (the results are then incomplete).
void launch_dense_fix(const DenseProb* d_probs, const uint32_t* ovf_n, const DenseOvf* ovf, uint32_t ovf_cap,
                      uint32_t* status, cudaStream_t st);

// Heavy features of sparse levels.  A feature held by many sequences costs
// about L^2 / 2 pair updates on the sparse route (L = its entries) but only
// one column of a dense contraction on the tensor cores.  After a sparse
// level's run-length pass, features with at least T entries whose counts
// are all <= 16 get a column of the (dataset, level)'s matrix A (e4m3,
// n_pad rows); their entries are flagged (kHeavyBit in efe) so that the
// on-chip accumulation skips them, and the dense GEMM adds A A^T to C_m.
// Which features go dense changes no result.
constexpr uint32_t kHeavyBit = 0x80000000u;
struct HeavyProb {
  uint8_t* A;          // n_pad x stride bytes
  uint32_t* ncols;     // columns handed out so far (may run past cap)
  uint32_t* maxc;      // largest count in A (for the GEMM's exact rounds)
  uint64_t stride;     // row stride of A in bytes (a multiple of 128)
  uint32_t cap;        // columns available (<= stride)
  uint32_t T;          // threshold on a feature's entries
  uint32_t n, n_pad;   // sequences; rows of A
  uint32_t prob;       // index of the GEMM's DenseProb record
  uint32_t pad;
};
// One heavy feature: entries [fs, fs + L) of the pool at `pool`, column col
// of heavy problem hp.
struct HeavyItem {
  uint64_t pool;
  uint32_t fs, L, col, hp;
  uint32_t pad[2];
};
// Per tile of a run-length chunk: features starting in the tile's entry
// range that qualify are appended to items[*nitems++] (nitems never
// exceeds the sum of the caps).  hmap[ds * levels + level] is the heavy
// problem of a (dataset, level) or kNone.
void launch_heavy_mark(const SegDesc* segs, const uint32_t* tile_seg, uint32_t ntiles,
                       const uint32_t* segtot, const uint32_t* mask_level, const uint32_t* hmap,
                       uint32_t levels, const HeavyProb* hprobs, const uint32_t* eseq,
                       const uint32_t* efe, HeavyItem* items, uint32_t* nitems, cudaStream_t st);
// Zeroes the used columns (rounded up to 128) of every heavy problem's A
// and sets the GEMM records' column counts; adds the columns and the
// upper-triangle flops to work[0], work[1].
void launch_heavy_zero(const HeavyProb* hprobs, uint32_t nh, uint32_t max_rows, DenseProb* dprobs,
                       unsigned long long* work, cudaStream_t st);
// Writes the listed features' counts into A and flags their entries.
void launch_heavy_scatter(const HeavyProb* hprobs, const HeavyItem* items, const uint32_t* nitems,
                          uint32_t* eseq, uint32_t* efe, int nsm, cudaStream_t st);

// Plain per-mask path (Alg. 1 as written: countAndUpdate straight into the
// global C_m with atomics, then inclusion-exclusion).
void launch_pairs_global(const uint32_t* segtot_E, const uint32_t* eseq,
                         const uint32_t* efe, uint32_t G, uint32_t* Cm,
                         uint32_t n, uint32_t* status, cudaStream_t st);
void launch_ie_combine(const DsInfo* d_ds, const uint32_t* C, uint32_t n,
                       const AccParams& coef, cudaStream_t st);

}  // namespace gk
