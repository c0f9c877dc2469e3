// Shared device-side definitions of the GaKCo engine (sm_103a).
//
// Terminology follows the paper (GaKCo, arXiv 1704.07468, Table 1):
//   g-mer     one contiguous window of g symbols of a sequence (Eq. 5);
//   mask      one choice of m of the g positions to delete (Section 2.2,
//             step 3); level m has C(g, m) masks, c_gk masks in total;
//   feature   one distinct (g-m)-mer of a mask, i.e. one run of equal keys
//             after sorting (Section 2.2, step 2);
//   entry     one (feature, sequence) pair with its count c > 0, i.e. one
//             nonzero of the per-mask count matrix F.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gk {

constexpr uint32_t kNone = 0xFFFFFFFFu;   // "no entry" marker
// Window slot of a feature held by one sequence: kSingleTag | count (entry
// indices stay below 2^31, kNone has bits 16..30 set).
constexpr uint32_t kSingleTag = 0x80000000u;
__host__ __device__ constexpr bool is_single(uint32_t v) { return (v >> 16) == (kSingleTag >> 16); }
constexpr int kMaxRuns = 16;              // kept-position runs per mask
constexpr int kMaxLevels = 16;            // M + 1 <= kMaxLevels
constexpr int kSortThreads = 256;         // threads of the sort / RLE blocks
constexpr int kSortIpt = 16;              // items per thread
constexpr int kTile = kSortThreads * kSortIpt;  // elements per tile
constexpr uint32_t kRecWords = 8;          // words of a run-length tile record
constexpr int kMaxRadixBits = 11;        // widest sort digit

// How to cut the kept positions of one mask out of a packed g-mer key.
// The full key holds symbol p of the window in bits
// [b*(g-1-p), b*(g-p)).  The masked key stands for the kept symbols in
// position order, so equal masked keys <=> equal (g-m)-mers:
//  - runs mode (fold == 0): the kept symbols' b-bit fields concatenated;
//    consecutive kept positions form a run that moves with one shift and
//    one mask;
//  - fold mode (fold == sigma, used when sigma is not a power of two): the
//    kept symbols as the digits of a base-sigma number, which needs
//    ceil(log2(sigma^(g-m))) bits instead of b(g-m) (e.g. 6 protein or text
//    symbols fit 32 bits).
struct MaskDesc {
  uint32_t level;               // m = number of deleted positions
  uint32_t nruns;
  uint32_t kbits;               // bits of the masked key
  uint32_t fold;                // 0: runs mode; else the base (sigma)
  uint32_t sr[kMaxRuns];        // right shift of the run in the full key
  uint32_t sl[kMaxRuns];        // left shift of the run in the masked key
  uint64_t msk[kMaxRuns];       // run mask after the right shift
  uint32_t nkeep;               // fold mode: kept positions
  uint32_t symmask;             // fold mode: (1 << b) - 1
  uint8_t ksh[64];              // fold mode: right shift of each kept symbol, in order
};

// The same in 32-bit arithmetic, for full keys of at most 32 bits (every
// shift is then below 32 and every run mask fits 32 bits).
__device__ __forceinline__ uint32_t masked_key32(uint32_t full, const MaskDesc& md) {
  uint32_t k = 0;
  if (md.fold) {
    for (uint32_t j = 0; j < md.nkeep; ++j) k = k * md.fold + ((full >> md.ksh[j]) & md.symmask);
    return k;
  }
  for (uint32_t r = 0; r < md.nruns; ++r) k |= ((full >> md.sr[r]) & (uint32_t)md.msk[r]) << md.sl[r];
  return k;
}

__device__ __forceinline__ uint64_t masked_key(uint64_t full,
                                               const MaskDesc& md) {
  uint64_t k = 0;
  if (md.fold) {
    for (uint32_t j = 0; j < md.nkeep; ++j) k = k * md.fold + ((full >> md.ksh[j]) & md.symmask);
    return k;
  }
  for (uint32_t r = 0; r < md.nruns; ++r)
    k |= ((full >> md.sr[r]) & md.msk[r]) << md.sl[r];
  return k;
}

// One (dataset, mask) sort segment.
struct SegDesc {
  uint64_t base;     // element offset of the segment in the chunk buffers
  uint64_t pool;     // offset of the segment in the per-mask pools
                     //   (= mask * G_total + window offset of the dataset)
  uint64_t hist;     // offset of its digit x tile counters
  uint32_t G;        // elements = windows of the dataset
  uint32_t win0;     // first global window of the dataset
  uint32_t mask;     // mask index
  uint32_t tile0;    // first tile (chunk-global numbering)
  uint32_t ntiles;
  uint32_t ds;       // dataset index (into the DsPack records)
};

// Per-dataset description used by the accumulation and finishing kernels.
struct DsInfo {
  const uint32_t* woff;   // n + 1 window offsets (dataset-local)
  int32_t* K;             // n x n int32 kernel (row-major)
  int32_t* Nm;            // (M+1) x n x n mismatch profiles, or null
  double* Khat;           // n x n normalised kernel, or null
  double* rinv;           // n: 1 / sqrt(K(x, x)), 0 when K(x, x) = 0
  uint32_t* C;            // (M+1) x n x n cumulative profiles (batched engine)
  uint64_t win0;          // first global window
  uint32_t n;
  uint32_t tile0;         // first 32x32 finishing tile of this dataset
  uint32_t seq0;          // first global sequence
  uint32_t pad;
};

// Error bits raised by kernels into the context's device status word.
enum : uint32_t {
  kErrKneCM = 1u,          // sum_m h_m N_m != C_M (must never happen)
  kErrBadEntry = 2u,       // entry index out of range
  kErrBadCode = 4u,        // a symbol >= sigma in the input
  kErrTimeout = 8u,        // a bounded wait in a pipelined kernel ran out
  kErrDenseOverflow = 16u, // the dense overflow list ran out of room
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace gk
