// Host side of the engine: the C ABI of include/gakco.h, input validation,
// the work plan, device memory, CUDA-graph replay, timing, the resident
// training index for cross kernels, and the serving loop.
//
// The work of one Gram call (Alg. 1 of GaKCo, arXiv 1704.07468):
//   1. pack every window of every dataset into a full g-mer key;
//   2. for every level m and mask, sort the masked keys and count runs
//      (batched: all (dataset, mask) segments of a chunk per launch);
//   3. accumulate rows of C_0..C_M on chip, group by group of masks;
//   4. apply Eq. 9 and Eq. 7, mirror the symmetric result and normalise.
// The plain engine instead runs one (dataset, mask) segment per launch and
// applies countAndUpdate with global atomics, as the paper states it.
//
// Every pipeline step runs on a Work: a stream plus the device buffers it
// needs.  The context owns one for its synchronous calls; each serving slot
// owns its own, so requests in different slots overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "gakco.h"
#include "launch.h"

using namespace gk;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Timed {
  const char* name;
  cudaEvent_t a, b;
};

struct Chunk {
  uint32_t level;
  uint32_t seg_first, nseg;
  uint32_t tile_first, ntiles;
  uint64_t elems;
  uint64_t hist_elems;
  bool wide;
  std::vector<std::pair<int, int>> passes;  // (shift, bits)
  uint64_t pass0 = 0;                       // plan-wide number of the chunk's first pass
};

struct DsHost {
  const uint8_t* codes;     // device
  const int64_t* off;       // host
  int32_t n;
  int32_t* K;
  double* Khat;
  int32_t* Nm;
  std::vector<uint32_t> woff;
  uint64_t G;
  uint64_t win0;
  uint32_t seq0;
  uint32_t tile0;
};

uint64_t binom(int n, int r) {
  if (r < 0 || r > n) return 0;
  uint64_t v = 1;
  for (int i = 1; i <= r; ++i) v = v * (uint64_t)(n - r + i) / (uint64_t)i;
  return v;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const uint8_t* b = (const uint8_t*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Device buffers and stream of one pipeline instance.
struct Work {
  cudaStream_t cs = nullptr;
  cudaStream_t cs2 = nullptr;                      // second branch of a Gram call
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_heavy = nullptr, ev_sparse = nullptr;
  DevBuf fullkey, wid, ewin, eseq, efe, keyA, keyB, valA, valB, hist, tcnt, segtot, estart,
      etseq, efid, fstart, tables, codes, outK, outKhat, outNm, rinv, status, Cplain, Cacc, ea, eb,
      Cd, Cx, Adense, dmaxc, dovf, outF, trec, Aheavy, hctr, hlist, dtot, osst, osctr, oscnt;
  void* h_tables = nullptr;
  size_t h_tables_cap = 0;
  void* h_status = nullptr;
  void* h_io = nullptr;  // pinned staging of a serving slot
  size_t h_io_cap = 0;
  void* h_out = nullptr;  // pinned staging of large host outputs (two chunks)
  size_t h_out_cap = 0;
  cudaEvent_t ev_out[2] = {nullptr, nullptr};
  int64_t launches = 0;
  bool dense_overflow = false;  // the last run's dense overflow list ran out of room
  std::string err;
  double pairs = 0, entries = 0, windows = 0;
  double heavy_cols = 0, heavy_flops = 0;  // heavy-feature columns and their GEMM flops
  double rle_entries = 0;                   // (feature, sequence) entries the run-length pass emitted

  std::vector<DevBuf*> all() {
    return {&fullkey, &wid, &ewin,   &eseq,  &efe,  &keyA,  &keyB,  &valA,    &valB,
            &hist,    &tcnt,    &segtot, &estart, &etseq, &efid, &fstart, &tables, &codes,
            &outK,    &outKhat, &outNm,  &rinv,  &status, &Cplain, &Cacc, &ea,    &eb,
            &Cd,      &Cx,      &Adense, &dmaxc,  &dovf,  &outF, &trec, &Aheavy, &hctr, &hlist, &dtot,
            &osst,    &osctr,   &oscnt};
  }
  size_t bytes() {
    size_t s = 0;
    for (DevBuf* b : all()) s += b->cap;
    return s;
  }
};

// Resident index of the fitted training set.
struct Train {
  bool ok = false;
  int32_t n = 0;
  uint64_t G = 0;
  std::vector<uint32_t> woff;
  DevBuf ukey, ufirst, eseq, nfeat, diagC, rinv;
  DevBuf tcodes;               // the training codes (for adding sequences)
  std::vector<int64_t> toff;   // their offsets
  // SVM coefficients alpha_i y_i for decision values (Eq. 1), if set.
  DevBuf svm;
  double svm_bias = 0;
  int svm_kind = 0;
  bool svm_ok = false;
};

struct Request {
  uint64_t ticket = 0;
  std::vector<uint8_t> codes;
  std::vector<int64_t> off;
  int32_t nt = 0;
  uint64_t windows = 0;
  int32_t* K = nullptr;     // caller host buffers
  double* Khat = nullptr;
  double* F = nullptr;      // SVM decision values, or null
  int rc = 1;               // 1 pending, 0 done, < 0 error
  std::string err;
  double t_submit = 0, t_done = 0;
};

struct Slot {
  Work w;
  std::vector<Request*> batch;
  std::vector<int32_t> row0;
  int32_t nt = 0;
  bool busy = false;
  std::atomic<bool> gpu_done{false};
  size_t k_off = 0, kh_off = 0, f_off = 0;  // output offsets in the pinned staging
};

}  // namespace

struct gakco_ctx {
  int sigma = 0, g = 0, k = 0, M = 0, bits = 0;
  std::vector<MaskDesc> masks;
  std::vector<uint32_t> mask_level;
  int lkbits[kMaxLevels] = {};  // masked-key bits of each level
  uint32_t h[kMaxLevels] = {};
  uint32_t ie[kMaxLevels][kMaxLevels] = {};
  uint32_t maxC = 0;  // max_m C(g, m), m <= M

  // options
  int engine = 0;
  int radix_bits = 8;
  int level_bits[kMaxLevels] = {};  // per-level digit width (0: radix_bits)
  int64_t chunk_elems = (int64_t)1 << 26;
  int use_graph = 1;
  int accum_threads = 256;
  int profile = 0;
  int64_t smem_cols = 0;
  std::atomic<int64_t> fail_alloc_after{0};
  int64_t group_bytes = (int64_t)128 << 20;
  int serve_slots = 3;
  int64_t serve_max_seqs = 512;
  int64_t serve_max_windows = (int64_t)1 << 19;
  int64_t serve_mem_bytes = 0;  // 0: no budget
  int dense = 0;                            // 0 off, 1 cost model, 2 every eligible level
  int64_t dense_bytes = (int64_t)16 << 30;  // A matrices per dense wave (capped at create)
  int64_t dense_overflow = 32768;           // overflow-list entries per dense wave
  // Columns of one dense problem (a run of masks of one level): long enough
  // to amortise a tile's epilogue, short enough that a level yields many
  // tiles and that concurrent tiles stay within one L2-sized window of A.
  int64_t dense_run_cols = 131072;
  int kernel_only = 0;  // 1: compute level M alone when N_m is not requested (K = C_M)
  int overlap = 1;      // 1: dense and sparse levels of a Gram call run on two streams
  int dense_sms = 0;    // CTAs of the dense GEMM (0: one per SM)
  int sort_mode = 0;    // 0: upsweep / digit scans / downsweep per pass; 1: onesweep
  int accum_variant = 0;  // how the accumulation walks short entry ranges (k_accum.cu)
  int rle_items = 16;     // elements per thread of the Gram run-length kernels (16 or 8)
  int dense_late = 0;     // 1: the GEMM waits for the sparse sort / run-length passes
  int dense_split = -1;   // cut the GEMM's partial last wave into K-parts: 1 always, 0 never,
                          // -1 when no sparse level runs beside the GEMM
  int64_t dense_round_sum = kDenseExactSum;  // bound on a GEMM round's partial sums
  int64_t dense_wait_cycles = 0;             // GEMM role-wait limit (0: default)
  // Heavy features of sparse levels go to the tensor cores: threshold on a
  // feature's entries in thousandths of the dataset's sequences (0: off),
  // and the bytes of their count matrices (capped at create).
  int heavy = 0;
  // Host outputs: -1 (default) copies straight into the caller's buffers
  // where the GPU uses the host page tables for pageable memory, else
  // through pinned staging; 0 = always staging, 1 = always direct.
  int direct_d2h = -1;
  bool pageable_ats = false;
  int64_t heavy_bytes = (int64_t)4 << 30;

  std::string err;
  int device = 0;
  int nsm = 0;
  size_t smem_optin = 0;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  Work main;

  cudaGraphExec_t gexec = nullptr;
  uint64_t gkey = 0;

  int64_t last_launches = 0, last_mask_passes = 0;
  int last_replay = 0;
  double last_pairs = 0, last_entries = 0, last_windows = 0;
  double last_heavy_cols = 0, last_heavy_flops = 0, last_rle_entries = 0;
  // Work figures of the last plan (kept for graph replays).
  double plan_dense_probs = 0, plan_dense_flops = 0, plan_dense_issued = 0, plan_dense_bytes = 0,
         plan_sort_bytes = 0, plan_rle_bytes = 0, plan_pack_bytes = 0, plan_combine_bytes = 0;
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> timings;

  Train train;
  Train train_add, train_merged;  // index of added sequences; merge target (swapped in)

  // serving
  std::mutex mu;
  std::condition_variable cv;
  std::thread dispatcher;
  bool serving = false, stopping = false;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> requests;
  std::vector<std::unique_ptr<Slot>> slots;
  uint64_t next_ticket = 1;
  int64_t served_batches = 0, served_requests = 0;
};

namespace {

int fail(gakco_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
  return code;
}

int wfail(Work& w, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  w.err = buf;
  return code;
}

int wcuda(Work& w, cudaError_t e, const char* what) {
  cudaGetLastError();
  return wfail(w, GAKCO_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Copies a Work's error into the context's message.
int ret(gakco_ctx* c, Work& w, int rc) {
  if (rc != GAKCO_OK) c->err = w.err;
  return rc;
}

int ensure(gakco_ctx* c, Work& w, DevBuf& b, size_t bytes, const char* what) {
  if (bytes <= b.cap) return GAKCO_OK;
  int64_t left = c->fail_alloc_after.load();
  while (left > 0 && !c->fail_alloc_after.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 1) return wfail(w, GAKCO_E_OOM, "injected allocation failure (%s, %zu bytes)", what, bytes);
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = align_up(std::max(bytes, (size_t)256), 256);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return wfail(w, GAKCO_E_OOM, "cudaMalloc(%s, %zu bytes): %s", what, want, cudaGetErrorString(e));
  }
  b.cap = want;
  return GAKCO_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

void release_work(Work& w) {
  if (w.cs) cudaStreamSynchronize(w.cs);
  if (w.cs2) cudaStreamSynchronize(w.cs2);
  if (w.cs2) cudaStreamDestroy(w.cs2);
  if (w.ev_fork) cudaEventDestroy(w.ev_fork);
  if (w.ev_join) cudaEventDestroy(w.ev_join);
  if (w.ev_heavy) cudaEventDestroy(w.ev_heavy);
  if (w.ev_sparse) cudaEventDestroy(w.ev_sparse);
  w.cs2 = nullptr;
  w.ev_fork = w.ev_join = w.ev_heavy = w.ev_sparse = nullptr;
  for (DevBuf* b : w.all()) release(*b);
  if (w.h_tables) cudaFreeHost(w.h_tables);
  if (w.h_status) cudaFreeHost(w.h_status);
  if (w.h_io) cudaFreeHost(w.h_io);
  if (w.h_out) cudaFreeHost(w.h_out);
  for (cudaEvent_t& e : w.ev_out)
    if (e) cudaEventDestroy(e), e = nullptr;
  w.h_out = nullptr;
  w.h_out_cap = 0;
  if (w.cs) cudaStreamDestroy(w.cs);
  w.h_tables = w.h_status = w.h_io = nullptr;
  w.cs = nullptr;
}

int init_work(Work& w) {
  cudaError_t e = cudaStreamCreateWithFlags(&w.cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.cs2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_heavy, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_sparse, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&w.h_status, 128);
  if (e != cudaSuccess) return wcuda(w, e, "work set-up");
  return GAKCO_OK;
}

int ensure_pinned(Work& w, void*& p, size_t& cap, size_t bytes, const char* what) {
  if (bytes <= cap) return GAKCO_OK;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  const size_t want = align_up(std::max(bytes, (size_t)1 << 16), 1 << 16);
  cudaError_t e = cudaMallocHost(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return wfail(w, GAKCO_E_OOM, "cudaMallocHost(%s, %zu): %s", what, want, cudaGetErrorString(e));
  }
  cap = want;
  return GAKCO_OK;
}

struct Xfer {
  void* dst;        // caller host buffer
  const void* src;  // device
  size_t bytes;
};

// First touch of large caller buffers (one write per 4 KiB) by host
// threads, started before the GPU work and joined before the copies: where
// the GPU reaches pageable memory through the host page tables, copying
// into touched pages runs at DMA speed, and the page faults of fresh
// buffers are taken by these threads while the GPU computes.
class PageTouch {
 public:
  PageTouch(bool on, const std::vector<Xfer>& xs) {
    size_t total = 0;
    for (const Xfer& x : xs) total += x.bytes;
    if (!on || total < ((size_t)8 << 20)) return;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nthr = std::min(16u, hw);
    try {
      for (unsigned t = 0; t < nthr; ++t)
        th_.emplace_back([xs, t, nthr] {
          for (const Xfer& x : xs) {
            const size_t pages = (x.bytes + 4095) / 4096, per = (pages + nthr - 1) / nthr;
            volatile uint8_t* b = (volatile uint8_t*)x.dst;
            for (size_t pg = t * per; pg < std::min(pages, (t + 1) * per); ++pg) b[pg * 4096] = 0;
          }
        });
    } catch (...) {
      // No threads to spare: the copies then take the page faults themselves.
    }
  }
  void wait() {
    for (std::thread& t : th_) t.join();
    th_.clear();
  }
  ~PageTouch() { wait(); }

 private:
  std::vector<std::thread> th_;
};

// Whether host outputs are copied straight into the caller's buffers.
bool direct_copies(const gakco_ctx* c) { return c->direct_d2h == 1 || (c->direct_d2h < 0 && c->pageable_ats); }

// Device results -> caller host buffers.  `direct`: one copy per buffer
// straight into the caller's (touched, see PageTouch) memory.  Otherwise
// large outputs go through two pinned 32 MiB staging chunks: the copy
// engine fills one chunk while several host threads move the previous one
// into the caller's (pageable) memory, instead of the driver's own small
// bounce buffers.
int copy_to_host(Work& w, const std::vector<Xfer>& xs, bool direct) {
  size_t total = 0;
  for (const Xfer& x : xs) total += x.bytes;
  cudaError_t e = cudaSuccess;
  if (direct || total < ((size_t)8 << 20)) {
    for (const Xfer& x : xs)
      if (x.bytes && e == cudaSuccess) e = cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDeviceToHost, w.cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w.cs);
    return e == cudaSuccess ? GAKCO_OK : wcuda(w, e, "copy results to host");
  }
  constexpr size_t kChunk = (size_t)32 << 20;
  int rc = ensure_pinned(w, w.h_out, w.h_out_cap, 2 * kChunk, "output staging");
  if (rc != GAKCO_OK) return rc;
  for (cudaEvent_t& ev : w.ev_out)
    if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return wcuda(w, e, "output staging events");
  struct Piece {
    uint8_t* dst;
    const uint8_t* src;
    size_t n;
  };
  std::vector<Piece> ps;
  for (const Xfer& x : xs)
    for (size_t o = 0; o < x.bytes; o += kChunk)
      ps.push_back({(uint8_t*)x.dst + o, (const uint8_t*)x.src + o, std::min(kChunk, x.bytes - o)});
  uint8_t* stage = (uint8_t*)w.h_out;
  auto issue = [&](size_t i) {
    uint8_t* slot = stage + (i & 1) * kChunk;
    cudaError_t r = cudaMemcpyAsync(slot, ps[i].src, ps[i].n, cudaMemcpyDeviceToHost, w.cs);
    if (r == cudaSuccess) r = cudaEventRecord(w.ev_out[i & 1], w.cs);
    return r;
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned nthr = std::min(8u, std::max(1u, hw / 2));
  e = issue(0);
  for (size_t i = 0; i < ps.size() && e == cudaSuccess; ++i) {
    if (i + 1 < ps.size() && (e = issue(i + 1)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(w.ev_out[i & 1])) != cudaSuccess) break;
    const uint8_t* slot = stage + (i & 1) * kChunk;
    uint8_t* dst = ps[i].dst;
    const size_t n = ps[i].n, part = (n + nthr - 1) / nthr;
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nthr; ++t) {
      const size_t a = std::min(n, t * part), b = std::min(n, (t + 1) * part);
      if (a >= b) continue;
      try {
        th.emplace_back([dst, slot, a, b] { memcpy(dst + a, slot + a, b - a); });
      } catch (...) {
        memcpy(dst + a, slot + a, b - a);  // no thread to spare: copy here
      }
    }
    memcpy(dst, slot, std::min(n, part));
    for (std::thread& t : th) t.join();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(w.cs);
  return e == cudaSuccess ? GAKCO_OK : wcuda(w, e, "copy results to host");
}

void drop_graph(gakco_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey = 0;
}

// Kernel-launch bracket: counts launches and, when profiling the context's
// own Work, records events around them on its stream.
struct Bracket {
  gakco_ctx* c;
  Work& w;
  const char* name;
  size_t ia = 0;
  bool on;
  Bracket(gakco_ctx* c_, Work& w_, const char* n_, int count)
      : c(c_), w(w_), name(n_), on(c_->profile && &w_ == &c_->main) {
    w.launches += count;
    if (on) {
      while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
      }
      ia = c->ev_used;
      c->ev_used += 2;
      cudaEventRecord(c->ev_pool[ia], w.cs);
    }
  }
  ~Bracket() {
    if (on) {
      cudaEventRecord(c->ev_pool[ia + 1], w.cs);
      c->timed.push_back({name, c->ev_pool[ia], c->ev_pool[ia + 1]});
    }
  }
};

// One dense problem (see DenseProb) before its device addresses are known.
struct DenseHost {
  uint32_t ds, level, mfirst, mcount, n, n_pad, key_bits, row0;
  uint64_t ld, a_off;  // columns; byte offset of A in the A buffer
  uint32_t hidx = 0;   // heavy problem index (when heavy)
  uint32_t nsib = 0;   // problems of its (dataset, level)
  bool sole = false;   // its wave's run holds every problem of the (dataset, level)
  bool heavy = false;  // heavy-feature matrix: ld is its column capacity, the
                       // columns in use are set on the device
};

// A heavy-feature problem of one sparse (dataset, level).
struct HeavyHost {
  uint32_t ds, level, n, n_pad, T, prob;
  uint64_t cap, a_off;  // columns (= row stride); byte offset in the heavy A buffer
};

struct DenseWave {
  uint32_t p0, np;       // problems
  uint32_t t0, nt;       // tiles
  uint32_t rows;         // A rows of the wave (the scatter grid)
  uint64_t elems;        // A bytes of the wave
};



struct Plan {
  std::vector<DsHost> ds;
  uint64_t gtot = 0;
  uint32_t nseq = 0;
  uint32_t nmax = 0;
  std::vector<Chunk> chunks;
  std::vector<SegDesc> segs;
  std::vector<uint32_t> tile_seg;
  std::vector<uint32_t> items;
  uint32_t ftiles = 0;
  uint64_t max_chunk_elems = 0, max_chunk_nseg = 0, max_chunk_tiles = 0, max_hist = 0;
  uint64_t total_passes = 0;  // sort passes of all chunks
  bool any_wide = false;
  uint32_t ncols = 0;
  size_t acc_smem = 0;
  int acc_blocks = 0;
  uint64_t c_elems = 0;
  std::vector<uint32_t> seg_ds;  // dataset of each segment
  bool want_nm = false, want_khat = false;
  // First level computed: M when only the kernel is wanted (K = C_M, so
  // C_0..C_{M-1} may stay zero: Eq. 9 then gives N_M = C_M and Eq. 7
  // K = h_M C_M = C_M), else 0.
  int first_level = 0;
  // Masks computed: [mask_lo, mask_hi) in level order (all by default; a
  // slice for a partial Gram whose C_0..C_M one rank of a sharded
  // computation adds), and where a partial call leaves its C.
  uint32_t mask_lo = 0, mask_hi = 0xFFFFFFFFu;
  uint32_t* partial_C = nullptr;
  // Dense (tensor-core) levels: flags per (dataset, level), problems,
  // waves of problems whose A matrices share the A buffer, GEMM tiles.
  std::vector<uint8_t> dense;
  std::vector<DenseHost> dprobs;
  std::vector<DenseWave> dwaves;
  std::vector<uint32_t> dtiles;
  uint64_t dense_abytes = 0;
  // Heavy features: problems, (dataset, level) -> problem map, GEMM tiles
  // [heavy_t0, heavy_t0 + heavy_nt) of dtiles.
  std::vector<HeavyHost> heavy;
  std::vector<uint32_t> hmap;
  std::vector<uint8_t> heavy_level;  // levels with a heavy problem
  uint32_t heavy_t0 = 0, heavy_nt = 0, heavy_rows = 0;
  uint64_t heavy_abytes = 0, heavy_list = 0;
  size_t o_hprobs = 0, o_hmap = 0;
  double dense_flops = 0;         // upper triangle of A A^T, unpadded: 2 mcount S n(n+1)/2 per problem
  double dense_issued = 0;        // what the 128 x 256 tiles issue, padding included
  double dense_bytes = 0;         // A written by the scatter
  double sort_bytes = 0;          // algorithmic bytes of every sort pass
  double rle_bytes = 0;           // run-length: (key, payload) read once + ewin written, per element
  double pack_bytes = 0;          // packing: symbols read once + full key and window id written
  double combine_bytes = 0;       // diag + combine: C_m upper triangles read, outputs written
  // device table offsets
  size_t o_masks, o_level, o_pack, o_info, o_segs, o_tiles, o_items, o_dprobs = 0, o_dtiles = 0, o_tmaps = 0;
  std::vector<size_t> o_coff, o_woff;

  bool is_dense(size_t d, int m, int M) const {
    return !dense.empty() && dense[d * (size_t)(M + 1) + (size_t)m];
  }
};

// Validate datasets and compute window offsets; fills p.ds.  `maxw_other`
// (windows of the longest sequence on the other side of a cross kernel, 0
// for a Gram) enters the int32 bound.
int plan_datasets(gakco_ctx* c, Work& w, Plan& p, int32_t nd, const uint8_t* const* codes,
                  const int64_t* const* off, const int32_t* n, int32_t* const* K,
                  double* const* Khat, int32_t* const* Nm, bool device, uint64_t maxw_other = 0) {
  if (nd < 0) return wfail(w, GAKCO_E_INVALID, "ndata must be >= 0");
  if (nd > 0 && (!codes || !off || !n)) return wfail(w, GAKCO_E_INVALID, "null dataset arrays");
  uint64_t wmax = 0;
  p.ds.resize(nd);
  for (int32_t d = 0; d < nd; ++d) {
    DsHost& D = p.ds[d];
    D.codes = codes[d];
    D.off = off[d];
    D.n = n[d];
    D.K = K ? K[d] : nullptr;
    D.Khat = Khat ? Khat[d] : nullptr;
    D.Nm = Nm ? Nm[d] : nullptr;
    if (D.n < 0 || D.n > 65535)
      return wfail(w, GAKCO_E_INVALID, "dataset %d: n = %d outside [0, 65535]", d, D.n);
    if (D.n > 0 && !D.off) return wfail(w, GAKCO_E_INVALID, "dataset %d: null offsets", d);
    if (device && D.n > 0 && !D.K)
      return wfail(w, GAKCO_E_INVALID, "dataset %d: device calls need a K buffer", d);
    D.woff.assign(D.n + 1, 0);
    uint64_t acc = 0;
    int64_t total = 0;
    for (int32_t x = 0; x < D.n; ++x) {
      const int64_t len = D.off[x + 1] - D.off[x];
      if (D.off[x] < 0 || len < 0)
        return wfail(w, GAKCO_E_INVALID, "dataset %d: offsets must be non-negative and non-decreasing", d);
      const uint64_t W = len >= c->g ? (uint64_t)(len - c->g + 1) : 0;
      if (W > 65535)
        return wfail(w, GAKCO_E_OVERFLOW, "dataset %d: sequence %d has %llu windows (at most 65535)", d, x,
                     (unsigned long long)W);
      wmax = std::max(wmax, W);
      acc += W;
      total += len;
      if (acc >= 0xFFFFFFFFull) return wfail(w, GAKCO_E_OVERFLOW, "dataset %d: 2^32 or more windows", d);
      D.woff[x + 1] = (uint32_t)acc;
    }
    if (D.n > 0 && total > 0 && !D.codes) return wfail(w, GAKCO_E_INVALID, "dataset %d: null codes", d);
    D.G = acc;
    D.win0 = p.gtot;
    D.seq0 = p.nseq;
    p.gtot += acc;
    p.nseq += (uint32_t)D.n;
    p.nmax = std::max<uint32_t>(p.nmax, (uint32_t)D.n);
    if (D.Nm) p.want_nm = true;
    if (D.Khat) p.want_khat = true;
  }
  // Every C_m(x, y) <= C(g, m) W_x W_y must stay below 2^31.
  const uint64_t wo = maxw_other ? maxw_other : wmax;
  const long double bound = (long double)c->maxC * (long double)wmax * (long double)wo;
  if (bound >= 2147483648.0L)
    return wfail(w, GAKCO_E_OVERFLOW,
                 "C(g,m) * W_max^2 = %.0Lf reaches 2^31 (W_max = %llu windows); int32 kernel would overflow",
                 bound, (unsigned long long)std::max(wmax, wo));
  return GAKCO_OK;
}

// Algorithmic bytes of packing and of the diagonal / combine tail: symbols
// read once, a full key (8 B) and a window id (4 B) written per window; the
// upper triangles of C_0..C_M read once and every requested output written.
void plan_io_bytes(gakco_ctx* c, Plan& p) {
  p.pack_bytes = 0;
  p.combine_bytes = 0;
  const double L = (double)(c->M + 1);
  for (const DsHost& D : p.ds) {
    if (D.n <= 0) continue;
    const double n = (double)D.n, nn = n * n;
    p.pack_bytes += (double)(D.off[D.n] - D.off[0]) + 12.0 * (double)D.G;
    p.combine_bytes += 4.0 * L * n * (n + 1.0) / 2.0 + (D.K ? 4.0 * nn : 0.0) + (D.Khat ? 8.0 * nn : 0.0) +
                       (D.Nm ? 4.0 * L * nn : 0.0);
  }
}

// Chunks of (dataset, mask) segments, all of one level per chunk.
void plan_chunks(gakco_ctx* c, Plan& p, bool plain) {
  p.sort_bytes = 0;
  p.total_passes = 0;
  const uint64_t limit = plain ? 0 : (uint64_t)std::max<int64_t>(c->chunk_elems, kTile);
  for (int m = p.first_level; m <= c->M; ++m) {
    const int kb = c->lkbits[m];
    const int rbits = c->level_bits[m] ? c->level_bits[m] : c->radix_bits;
    const int np = (kb + rbits - 1) / rbits;
    const int rb = (kb + np - 1) / np;
    std::vector<std::pair<int, int>> passes;
    for (int q = 0; q < np; ++q) passes.push_back({q * rb, std::min(rb, kb - q * rb)});
    const bool wide = kb > 32;
    p.any_wide |= wide;
    Chunk cur{};
    auto flush = [&]() {
      if (cur.nseg == 0) return;
      // Per element: the first pass reads the full key and the window id
      // and writes (key, payload); later passes read and write both.
      const double kbytes = wide ? 8.0 : 4.0;
      p.sort_bytes += (double)cur.elems * ((8.0 + 4.0 + kbytes + 4.0) + 2.0 * (kbytes + 4.0) * (np - 1));
      p.rle_bytes += (double)cur.elems * (kbytes + 4.0 + 4.0);
      cur.pass0 = p.total_passes;
      p.total_passes += cur.passes.size();
      p.chunks.push_back(cur);
      p.max_chunk_elems = std::max(p.max_chunk_elems, cur.elems);
      p.max_chunk_nseg = std::max<uint64_t>(p.max_chunk_nseg, cur.nseg);
      p.max_chunk_tiles = std::max<uint64_t>(p.max_chunk_tiles, cur.ntiles);
      p.max_hist = std::max(p.max_hist, cur.hist_elems);
    };
    auto fresh = [&]() {
      cur = Chunk{};
      cur.level = m;
      cur.seg_first = (uint32_t)p.segs.size();
      cur.tile_first = (uint32_t)p.tile_seg.size();
      cur.wide = wide;
      cur.passes = passes;
    };
    fresh();
    for (uint32_t mu = 0; mu < c->masks.size(); ++mu) {
      if ((int)c->mask_level[mu] != m || mu < p.mask_lo || mu >= p.mask_hi) continue;
      for (size_t d = 0; d < p.ds.size(); ++d) {
        const DsHost& D = p.ds[d];
        if (D.G == 0 || p.is_dense(d, m, c->M)) continue;
        if (cur.nseg > 0 && (plain || cur.elems + D.G > limit)) {
          flush();
          fresh();
        }
        SegDesc s{};
        s.base = cur.elems;
        s.pool = (plain ? 0 : (uint64_t)mu * p.gtot) + D.win0;
        s.hist = cur.hist_elems;
        s.G = (uint32_t)D.G;
        s.win0 = (uint32_t)D.win0;
        s.mask = mu;
        s.tile0 = cur.ntiles;
        s.ntiles = (uint32_t)((D.G + kTile - 1) / kTile);
        s.ds = (uint32_t)d;
        for (uint32_t t = 0; t < s.ntiles; ++t) p.tile_seg.push_back(cur.nseg);
        cur.ntiles += s.ntiles;
        cur.hist_elems += ((uint64_t)1 << rb) * s.ntiles;
        cur.elems += D.G;
        cur.nseg += 1;
        p.segs.push_back(s);
        p.seg_ds.push_back((uint32_t)d);
      }
    }
    flush();
  }
}

std::vector<uint32_t> level_firsts(gakco_ctx* c) {
  std::vector<uint32_t> lf(c->M + 2, 0);
  for (uint32_t mu = 0; mu < c->masks.size(); ++mu) lf[c->mask_level[mu] + 1] = mu + 1;
  for (int m = 1; m <= c->M + 1; ++m) lf[m] = std::max(lf[m], lf[m - 1]);
  return lf;
}

uint32_t smem_columns(gakco_ctx* c, uint32_t n) {
  const size_t avail = c->smem_optin > 2048 ? c->smem_optin - 1024 : 0;
  uint32_t ncols = (uint32_t)std::min<size_t>(avail / 4 - 1, 65535);
  if (c->smem_cols > 0) ncols = std::min<uint32_t>(ncols, (uint32_t)c->smem_cols);
  return std::max<uint32_t>(1, std::min<uint32_t>(ncols, std::max<uint32_t>(n, 1)));
}

// Work items of the accumulation kernels: (dataset, level, first mask, mask
// count, row, c0, c1).  The masks of a level are cut into groups whose
// entry arrays (`per_mask_bytes` each) fit `group_bytes`, so the rows
// processed together share an L2-resident working set; items go out group
// by group, most expensive rows first within a group.  `triangle` keeps
// only columns y >= x (Gram); `ncols_total` is the column count.
void add_items(gakco_ctx* c, std::vector<uint32_t>& items, uint32_t d, const std::vector<uint32_t>& woff,
               uint32_t nrows, uint32_t ncols_total, uint32_t ncols, double per_mask_bytes,
               bool triangle, const Plan* skip = nullptr) {
  struct Row {
    double cost;
    uint32_t x, c0, c1;
  };
  std::vector<Row> rows;
  for (uint32_t x = 0; x < nrows; ++x) {
    const double W = (double)(woff[x + 1] - woff[x]);
    if (W == 0) continue;  // its row of C stays zero (memset)
    for (uint32_t t0 = 0; t0 < ncols_total; t0 += ncols) {
      const uint32_t t1 = std::min<uint32_t>(ncols_total, t0 + ncols);
      if (triangle && t1 <= x) continue;
      const uint32_t c0 = triangle ? std::max<uint32_t>(x, t0) : t0;
      rows.push_back({W * (double)(t1 - c0) + W + (double)(t1 - c0), x, c0, t1});
    }
  }
  std::stable_sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) { return a.cost > b.cost; });
  const std::vector<uint32_t> lf = level_firsts(c);
  const uint32_t gmax =
      (uint32_t)std::max(1.0, std::floor((double)c->group_bytes / std::max(per_mask_bytes, 1.0)));
  for (int m = 0; m <= c->M; ++m) {
    if (skip && (m < skip->first_level || skip->is_dense(d, m, c->M))) continue;  // not needed / tensor cores
    uint32_t mf = lf[m], me = lf[m + 1];
    if (skip) {
      mf = std::max(mf, skip->mask_lo);
      me = std::min(me, skip->mask_hi);
    }
    if (me <= mf) continue;  // no mask of this level in the plan's slice
    const uint32_t mc = me - mf;
    const uint32_t ng = (mc + gmax - 1) / gmax;
    for (uint32_t gi = 0; gi < ng; ++gi) {
      const uint32_t a = mf + (uint32_t)((uint64_t)mc * gi / ng);
      const uint32_t b = mf + (uint32_t)((uint64_t)mc * (gi + 1) / ng);
      for (const Row& r : rows) {
        const uint32_t it[kItemWords] = {d, (uint32_t)m, a, b - a, r.x, r.c0, r.c1, 0};
        items.insert(items.end(), it, it + kItemWords);
      }
    }
  }
}

void plan_items(gakco_ctx* c, Plan& p) {
  const uint32_t ncols = smem_columns(c, p.nmax);
  p.ncols = ncols;
  p.acc_smem = 4 * ((size_t)ncols + 1);  // + the trash slot
  p.items.clear();
  for (size_t d = 0; d < p.ds.size(); ++d) {
    const DsHost& D = p.ds[d];
    if (D.n == 0) continue;
    add_items(c, p.items, (uint32_t)d, D.woff, (uint32_t)D.n, (uint32_t)D.n, ncols,
              12.0 * (double)std::max<uint64_t>(D.G, 1), true, &p);
  }
}

// Per-mask time estimates (seconds) of one level of one dataset on the
// sparse route (sort, run-length, pair updates) and on the dense route
// (scatter into A, tensor-core GEMM), from effective rates of the kernels.
bool dense_is_cheaper(gakco_ctx* c, const DsHost& D, uint32_t n_pad, int kb) {
  const double hbm = 6.0e12, updates = 1.0e12, tensor = 2.0e15;
  const double G = (double)D.G, S = std::ldexp(1.0, kb);
  const double passes = std::ceil((double)kb / (double)c->radix_bits);
  const double sparse = G * (passes * 16.0 + 48.0) / hbm + 0.5 * (G * G / S + G) / updates;
  const double rb = n_pad / 128.0, cb = std::ceil(n_pad / 256.0);
  const double tiles = rb * cb - std::floor(rb / 2.0) * std::ceil(rb / 2.0);
  const double dense = tiles * 128.0 * 256.0 * 2.0 * std::max(S, 128.0) / tensor + 3.0 * n_pad * S / hbm;
  return dense < sparse;
}

// Marks the (dataset, level) pairs that run on the tensor cores and cuts
// them into problems (runs of masks of at most kDenseRunCols columns whose
// A fits the wave budget), waves and upper-triangle output tiles, the
// tiles of a wave longest first.  A level qualifies when its masked keys
// have at most 16 bits and one mask's A fits the budget.
void plan_dense(gakco_ctx* c, Plan& p, bool plain) {
  const int L = c->M + 1;
  p.dense.assign(p.ds.size() * (size_t)L, 0);
  p.dprobs.clear();
  p.dwaves.clear();
  p.dtiles.clear();
  p.dense_abytes = 0;
  p.dense_flops = p.dense_issued = p.dense_bytes = 0;
  if (plain || c->dense == 0) return;
  const std::vector<uint32_t> lf = level_firsts(c);
  const uint64_t budget = (uint64_t)std::max<int64_t>(c->dense_bytes, 1);
  for (size_t d = 0; d < p.ds.size(); ++d) {
    const DsHost& D = p.ds[d];
    if (D.n == 0 || D.G == 0) continue;
    const uint32_t n_pad = (uint32_t)align_up((size_t)D.n, 128);
    for (int m = p.first_level; m <= c->M; ++m) {
      const int kb = c->lkbits[m];
      if (kb > 16) continue;
      const uint64_t S = (uint64_t)1 << kb;
      const uint64_t per_mask = (uint64_t)n_pad * S;
      if (per_mask > budget) continue;
      const uint32_t mf = std::max(lf[m], p.mask_lo), me = std::min(lf[m + 1], p.mask_hi);
      if (me <= mf) continue;  // no mask of this level in the plan's slice
      if (c->dense == 1 && !dense_is_cheaper(c, D, n_pad, kb)) continue;
      p.dense[d * L + m] = 1;
      const uint32_t mc = me - mf;
      const uint64_t by_mem = std::max<uint64_t>(1, budget / per_mask);
      // (A problem's row stays below 2^31 columns: the scatter indexes a
      // row's columns in 32-bit arithmetic.)
      const uint64_t by_cols =
          std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)c->dense_run_cols, (uint64_t)1 << 31) / S);
      const uint32_t gmax = (uint32_t)std::min<uint64_t>(mc, std::min(by_mem, by_cols));
      const uint32_t ng = (mc + gmax - 1) / gmax;
      for (uint32_t gi = 0; gi < ng; ++gi) {
        const uint32_t a = mf + (uint32_t)((uint64_t)mc * gi / ng);
        const uint32_t b = mf + (uint32_t)((uint64_t)mc * (gi + 1) / ng);
        DenseHost h{};
        h.ds = (uint32_t)d;
        h.level = (uint32_t)m;
        h.mfirst = a;
        h.mcount = b - a;
        h.n = (uint32_t)D.n;
        h.n_pad = n_pad;
        h.key_bits = (uint32_t)kb;
        h.ld = align_up((size_t)h.mcount * S, 128);
        h.nsib = ng;
        p.dprobs.push_back(h);
      }
    }
  }
  // Waves: consecutive problems whose A matrices fit the budget together.
  // A wave's macro tiles cover each run of its problems that shares one
  // (dataset, level); longest first, so the persistent CTAs finish together.
  // Each macro tile issues one 128 x 256 product per row half below n.
  auto sub_tiles = [](uint32_t I2, uint32_t, uint32_t n) {
    return (I2 * 256 < n ? 2 : 0) + (I2 * 256 + 128 < n ? 2 : 0);  // in 128 x 128 units
  };
  DenseWave wv{};
  // Cutting the partial last wave into K-parts pays only when no sparse
  // level runs beside the GEMM (otherwise the sparse branch fills the idle
  // SMs of that wave): auto (-1) splits when every level with work is dense.
  bool all_dense = true;
  for (size_t d = 0; d < p.ds.size(); ++d)
    for (int m = p.first_level; m <= c->M; ++m)
      if (p.ds[d].G > 0 && !p.is_dense(d, m, c->M) && std::min(lf[m + 1], p.mask_hi) > std::max(lf[m], p.mask_lo))
        all_dense = false;
  const bool split = c->dense_split == 1 || (c->dense_split == -1 && all_dense);
  auto close = [&]() {
    if (wv.np == 0) return;
    // Macro tiles per (dataset, level) run of problems, each sweeping all
    // of the run's columns (one epilogue per tile: tensor memory holds no
    // second accumulator pair to overlap more), longest first.
    struct Part {
      std::array<uint32_t, kDenseTileWords> w;
      double cost;
    };
    std::vector<Part> best;
    for (uint32_t g0 = wv.p0; g0 < wv.p0 + wv.np;) {
      uint32_t g1 = g0 + 1;
      while (g1 < wv.p0 + wv.np && p.dprobs[g1].ds == p.dprobs[g0].ds && p.dprobs[g1].level == p.dprobs[g0].level) ++g1;
      for (uint32_t j = g0; j < g1; ++j) p.dprobs[j].sole = (g1 - g0) == p.dprobs[j].nsib;
      const DenseHost& h = p.dprobs[g0];
      double stages = 0;
      for (uint32_t j = g0; j < g1; ++j) stages += (double)(p.dprobs[j].ld / 128);
      const uint32_t R = (h.n_pad + 255) / 256;
      for (uint32_t I2 = 0; I2 < R; ++I2)
        for (uint32_t J2 = I2; J2 < R; ++J2) {
          const int k = sub_tiles(I2, J2, h.n);
          if (k > 0) best.push_back({{g0, g1 - g0, I2, J2, 0u, (uint32_t)stages}, stages * k});
        }
      g0 = g1;
    }
    std::stable_sort(best.begin(), best.end(), [](const Part& x, const Part& y) { return x.cost > y.cost; });
    // The persistent CTAs take tiles b, b + C, ...: the tiles past the last
    // full multiple of C form a partial last wave.  Cut each of those into q
    // K-parts (q minimising the tail's length in tile units, ceil(r q / C) /
    // q, when the tail tiles cost the same), ordered part by part so that
    // concurrent CTAs still sweep the same columns of A.
    {
      const uint32_t C = (uint32_t)(c->dense_sms > 0 ? std::min(c->dense_sms, c->nsm) : c->nsm);
      const size_t T = best.size(), full = C ? T / C * C : T, r = T - full;
      bool equal = r > 0 && split;
      for (size_t i = full; i < T && equal; ++i) equal = best[i].cost == best[full].cost;
      if (equal && C > 0) {
        uint32_t q = 1;
        double span = 1.0;
        for (uint32_t cand = 2; cand <= 8; ++cand) {
          const double sp = std::ceil((double)r * cand / C) / cand;
          if (sp < span - 1e-9 && best[full].w[5] >= 16 * cand) span = sp, q = cand;
        }
        if (q > 1) {
          std::vector<Part> tail(best.begin() + full, best.end());
          best.resize(full);
          for (uint32_t part = 0; part < q; ++part)
            for (const Part& pt : tail) {
              Part x = pt;
              const uint32_t S = pt.w[5];
              x.w[4] = (uint32_t)((uint64_t)S * part / q);
              x.w[5] = (uint32_t)((uint64_t)S * (part + 1) / q);
              x.cost = pt.cost / q;
              best.push_back(x);
            }
        }
      }
    }
    wv.t0 = (uint32_t)(p.dtiles.size() / kDenseTileWords);
    for (const Part& pt : best) {
      p.dtiles.insert(p.dtiles.end(), pt.w.begin(), pt.w.end());
      const double cols = 128.0 * (double)(pt.w[5] - pt.w[4]);
      p.dense_issued += 2.0 * 128.0 * 128.0 * cols * sub_tiles(pt.w[2], pt.w[3], p.dprobs[pt.w[0]].n);
    }
    wv.nt = (uint32_t)best.size();
    p.dense_abytes = std::max<uint64_t>(p.dense_abytes, wv.elems);
    p.dwaves.push_back(wv);
  };
  for (uint32_t i = 0; i < (uint32_t)p.dprobs.size(); ++i) {
    DenseHost& h = p.dprobs[i];
    const uint64_t el = (uint64_t)h.n_pad * h.ld;
    if (wv.np > 0 && wv.elems + el > budget) {
      close();
      wv = DenseWave{};
    }
    if (wv.np == 0) wv.p0 = i;
    h.a_off = wv.elems;
    h.row0 = wv.rows;
    wv.elems += el;
    wv.rows += h.n_pad;
    wv.np++;
    p.dense_flops += 2.0 * (double)h.mcount * std::ldexp(1.0, (int)h.key_bits) * 0.5 * h.n * (h.n + 1.0);
    p.dense_bytes += (double)el;
  }
  close();
}

constexpr uint32_t kHeavyMinSeqs = 256;  // smaller datasets keep every feature sparse
constexpr uint32_t kHeavyMinT = 8;       // smallest entry threshold

// Heavy features (see HeavyProb): one problem per sparse (dataset, level)
// of a dataset with at least kHeavyMinSeqs sequences.  Its column capacity
// is a share of the byte budget in proportion to the most heavy features
// the level can hold (masks x windows / T), at most that number; its GEMM
// macro tiles follow the regular dense tiles, largest problems first.  A
// feature of the dataset is heavy when it has at least T = ceil(heavy n /
// 1000) entries (and at least kHeavyMinT); the break-even of a tensor-core
// column (n^2 flops) against L^2 / 2 pair updates lies near L = 0.02 n.
void plan_heavy(gakco_ctx* c, Plan& p, bool plain) {
  const int L = c->M + 1;
  p.heavy.clear();
  p.hmap.assign(p.ds.size() * (size_t)L, kNone);
  p.heavy_level.assign((size_t)L, 0);
  p.heavy_t0 = (uint32_t)(p.dtiles.size() / kDenseTileWords);
  p.heavy_nt = 0;
  p.heavy_rows = 0;
  p.heavy_abytes = p.heavy_list = 0;
  if (plain || c->heavy <= 0) return;
  const std::vector<uint32_t> lf = level_firsts(c);
  struct Cand {
    HeavyHost h;
    double most;
  };
  std::vector<Cand> cand;
  double wsum = 0;
  for (size_t d = 0; d < p.ds.size(); ++d) {
    const DsHost& D = p.ds[d];
    if ((uint64_t)D.n < kHeavyMinSeqs || D.G == 0 || D.G >= (uint64_t)kHeavyBit) continue;
    const uint32_t T =
        std::max<uint32_t>(kHeavyMinT, (uint32_t)(((uint64_t)c->heavy * (uint64_t)D.n + 999) / 1000));
    for (int m = p.first_level; m <= c->M; ++m) {
      if (p.is_dense(d, m, c->M)) continue;
      HeavyHost h{};
      h.ds = (uint32_t)d;
      h.level = (uint32_t)m;
      h.n = (uint32_t)D.n;
      h.n_pad = (uint32_t)align_up((size_t)D.n, 128);
      h.T = T;
      const uint32_t mf = std::max(lf[m], p.mask_lo), me = std::min(lf[m + 1], p.mask_hi);
      if (me <= mf) continue;
      const double most = (double)(me - mf) * (double)D.G / (double)T;
      cand.push_back({h, most});
      wsum += most;
    }
  }
  const double budget = (double)std::max<int64_t>(c->heavy_bytes, 0);
  std::vector<double> cost;
  for (const Cand& k : cand) {
    HeavyHost h = k.h;
    uint64_t cap = (uint64_t)(budget * k.most / wsum / (double)h.n_pad) / 128 * 128;
    cap = std::min<uint64_t>(cap, align_up((size_t)std::ceil(k.most), 128));
    cap = std::min<uint64_t>(cap, (uint64_t)1 << 30);
    if (cap < 128) continue;
    h.cap = cap;
    h.a_off = p.heavy_abytes;
    h.prob = (uint32_t)p.dprobs.size();
    p.heavy_abytes += align_up((size_t)(cap * h.n_pad), 128);
    p.heavy_list += cap;
    DenseHost q{};
    q.ds = h.ds;
    q.level = h.level;
    q.n = h.n;
    q.n_pad = h.n_pad;
    q.ld = cap;
    q.a_off = h.a_off;
    q.hidx = (uint32_t)p.heavy.size();
    q.heavy = true;
    p.dprobs.push_back(q);
    p.hmap[(size_t)h.ds * L + h.level] = (uint32_t)p.heavy.size();
    p.heavy_level[h.level] = 1;
    p.heavy_rows = std::max(p.heavy_rows, h.n_pad);
    p.heavy.push_back(h);
    cost.push_back(k.most);
  }
  struct Part {
    std::array<uint32_t, kDenseTileWords> w;
    double cost;
  };
  std::vector<Part> parts;
  for (size_t i = 0; i < p.heavy.size(); ++i) {
    const HeavyHost& h = p.heavy[i];
    const uint32_t R = (h.n_pad + 255) / 256;
    for (uint32_t I2 = 0; I2 < R; ++I2)
      for (uint32_t J2 = I2; J2 < R; ++J2)
        if (I2 * 256 < h.n)
          parts.push_back({{h.prob, 1u, I2, J2, 0u, 0xFFFFFFFFu},
                           cost[i] * (double)h.n * (I2 * 256 + 128 < h.n ? 2.0 : 1.0)});
  }
  std::stable_sort(parts.begin(), parts.end(), [](const Part& x, const Part& y) { return x.cost > y.cost; });
  for (const Part& pt : parts) p.dtiles.insert(p.dtiles.end(), pt.w.begin(), pt.w.end());
  p.heavy_nt = (uint32_t)parts.size();
}

struct Tables {
  std::vector<uint8_t> buf;
  size_t add(const void* src, size_t bytes, size_t align = 16) {
    const size_t o = align_up(buf.size(), align);
    buf.resize(o + bytes);
    if (bytes) memcpy(buf.data() + o, src, bytes);
    return o;
  }
  size_t reserve(size_t bytes, size_t align = 16) {
    const size_t o = align_up(buf.size(), align);
    buf.resize(o + bytes);
    return o;
  }
};

// Copy host tables into the Work's device table area through pinned memory.
int upload_tables(gakco_ctx* c, Work& w, Tables& t) {
  int rc = ensure(c, w, w.tables, t.buf.size(), "tables");
  if (rc != GAKCO_OK) return rc;
  if ((rc = ensure_pinned(w, w.h_tables, w.h_tables_cap, t.buf.size(), "tables")) != GAKCO_OK) return rc;
  // The pinned staging area may still feed an earlier copy.
  cudaError_t e = cudaStreamSynchronize(w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "stream sync before table upload");
  memcpy(w.h_tables, t.buf.data(), t.buf.size());
  e = cudaMemcpyAsync(w.tables.p, w.h_tables, t.buf.size(), cudaMemcpyHostToDevice, w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "table upload");
  return GAKCO_OK;
}

#define ENSURE(buf, bytes)                                                          \
  do {                                                                              \
    if ((rc = ensure(c, w, w.buf, (size_t)(bytes), #buf)) != GAKCO_OK) return rc; \
  } while (0)

// The onesweep sort takes digits of at most 8 bits (one look-back thread
// per digit) and at most kOsMaxPasses passes.
bool use_onesweep(const gakco_ctx* c) {
  return c->sort_mode == 1;
}

// Sort / run-length buffers for the plan's largest chunk.
int ensure_sort_buffers(gakco_ctx* c, Work& w, const Plan& p) {
  int rc;
  const uint64_t ce = p.max_chunk_elems;
  const size_t kbytes = p.any_wide ? 8 : 4;
  ENSURE(keyA, ce * kbytes);
  ENSURE(keyB, ce * kbytes);
  ENSURE(valA, ce * 4);
  ENSURE(valB, ce * 4);
  ENSURE(hist, p.max_hist * 4);
  ENSURE(dtot, (p.max_chunk_nseg << kMaxRadixBits) * 4);
  ENSURE(tcnt, p.max_chunk_tiles * 8);
  ENSURE(trec, p.max_chunk_tiles * kRecWords * 4);
  ENSURE(segtot, p.max_chunk_nseg * 8);
  const uint64_t te = ce + p.max_chunk_nseg + 1;
  ENSURE(estart, te * 4);
  ENSURE(etseq, te * 4);
  ENSURE(efid, te * 4);
  ENSURE(fstart, te * 4);
  ENSURE(status, 128);
  if (use_onesweep(c)) {
    ENSURE(osst, p.max_chunk_tiles * kOsRadix * 8);
    ENSURE(osctr, (p.total_passes + 1) * 4);
    ENSURE(oscnt, p.max_chunk_nseg * kOsMaxPasses * kOsRadix * 4);
  }
  return GAKCO_OK;
}

// Common tables: masks, levels, segments, tiles, items, per-dataset offsets
// and room for the DsPack / DsInfo records.
void add_common_tables(gakco_ctx* c, Plan& p, Tables& t) {
  p.o_masks = t.add(c->masks.data(), c->masks.size() * sizeof(MaskDesc));
  p.o_level = t.add(c->mask_level.data(), c->mask_level.size() * 4);
  p.o_segs = t.add(p.segs.data(), p.segs.size() * sizeof(SegDesc));
  p.o_tiles = t.add(p.tile_seg.data(), p.tile_seg.size() * 4);
  p.o_items = t.add(p.items.data(), p.items.size() * 4);
  p.o_coff.resize(p.ds.size());
  p.o_woff.resize(p.ds.size());
  for (size_t d = 0; d < p.ds.size(); ++d) {
    const DsHost& D = p.ds[d];
    p.o_coff[d] = D.n > 0 ? t.add(D.off, (D.n + 1) * 8) : t.reserve(8);
    p.o_woff[d] = t.add(D.woff.data(), D.woff.size() * 4);
  }
  p.o_pack = t.reserve(p.ds.size() * sizeof(DsPack));
  p.o_info = t.reserve(p.ds.size() * sizeof(DsInfo));
  if (!p.dprobs.empty()) {
    p.o_dprobs = t.reserve(p.dprobs.size() * sizeof(DenseProb));
    p.o_dtiles = t.add(p.dtiles.data(), p.dtiles.size() * 4);
    p.o_tmaps = t.reserve(p.dprobs.size() * kDenseTmapBytes, 64);
  }
  if (!p.heavy.empty()) {
    p.o_hprobs = t.reserve(p.heavy.size() * sizeof(HeavyProb));
    p.o_hmap = t.add(p.hmap.data(), p.hmap.size() * 4);
  }
}

// Dense problem records and their TMA descriptors, once the A buffer and
// the table area have device addresses.
int fill_dense(gakco_ctx* c, Work& w, Plan& p, Tables& t) {
  uint8_t* base = (uint8_t*)w.tables.p;
  std::vector<uint64_t> cacc(p.ds.size(), 0);
  for (size_t d = 1; d < p.ds.size(); ++d)
    cacc[d] = cacc[d - 1] + (uint64_t)(c->M + 1) * p.ds[d - 1].n * p.ds[d - 1].n;
  for (size_t i = 0; i < p.dprobs.size(); ++i) {
    const DenseHost& h = p.dprobs[i];
    const uint32_t nh = (uint32_t)p.heavy.size();
    DenseProb q{};
    q.A = (h.heavy ? (uint8_t*)w.Aheavy.p : (uint8_t*)w.Adense.p) + h.a_off;
    q.C = (uint32_t*)w.Cacc.p + cacc[h.ds] + (uint64_t)h.level * h.n * h.n;
    q.maxc = h.heavy ? (uint32_t*)w.hctr.p + nh + h.hidx : (uint32_t*)w.dmaxc.p + (size_t)h.ds * (c->M + 1) + h.level;
    q.tmap = base + p.o_tmaps + i * kDenseTmapBytes;
    q.ld = h.heavy ? 0 : h.ld;  // heavy: the columns in use, set on the device
    q.n = h.n;
    q.n_pad = h.n_pad;
    q.ds = h.ds;
    q.mfirst = h.mfirst;
    q.mcount = h.mcount;
    q.key_bits = h.key_bits;
    q.row0 = h.row0;
    q.sole = h.sole ? 1u : 0u;
    if (!h.heavy) {
      const std::vector<uint32_t>& wo = p.ds[h.ds].woff;
      uint64_t wmax = 0;
      for (size_t x = 0; x + 1 < wo.size(); ++x) wmax = std::max<uint64_t>(wmax, wo[x + 1] - wo[x]);
      const std::vector<uint32_t> lf = level_firsts(c);
      const uint64_t wm = wmax * (uint64_t)(lf[h.level + 1] - lf[h.level]);
      q.wmasks = wm <= 0xFFFFFFFFull ? (uint32_t)wm : 0u;
    }
    memcpy(t.buf.data() + p.o_dprobs + i * sizeof(DenseProb), &q, sizeof q);
    const int r = dense_encode_tmap(t.buf.data() + p.o_tmaps + i * kDenseTmapBytes, q.A, h.ld, h.n_pad);
    if (r != 0) return wfail(w, GAKCO_E_CUDA, "TMA descriptor of dense problem %zu failed (%d)", i, r);
  }
  for (size_t i = 0; i < p.heavy.size(); ++i) {
    const HeavyHost& h = p.heavy[i];
    HeavyProb r{};
    r.A = (uint8_t*)w.Aheavy.p + h.a_off;
    r.ncols = (uint32_t*)w.hctr.p + i;
    r.maxc = (uint32_t*)w.hctr.p + p.heavy.size() + i;
    r.stride = h.cap;
    r.cap = (uint32_t)h.cap;
    r.T = h.T;
    r.n = h.n;
    r.n_pad = h.n_pad;
    r.prob = h.prob;
    memcpy(t.buf.data() + p.o_hprobs + i * sizeof(HeavyProb), &r, sizeof r);
  }
  return GAKCO_OK;
}

// Fill the DsPack / DsInfo records once the table area's device address
// is known; returns the finishing-tile count.
uint32_t fill_records(gakco_ctx* c, Work& w, Plan& p, Tables& t, bool plain) {
  uint8_t* base = (uint8_t*)w.tables.p;
  double* rinv = (double*)w.rinv.p;
  uint64_t cacc = 0;
  uint32_t ftile = 0;
  for (size_t d = 0; d < p.ds.size(); ++d) {
    DsHost& D = p.ds[d];
    DsPack pk{};
    pk.codes = D.codes;
    pk.coff = (const int64_t*)(base + p.o_coff[d]);
    pk.woff = (const uint32_t*)(base + p.o_woff[d]);
    pk.win0 = D.win0;
    pk.n = (uint32_t)D.n;
    pk.seq0 = D.seq0;
    memcpy(t.buf.data() + p.o_pack + d * sizeof(DsPack), &pk, sizeof pk);
    DsInfo in{};
    in.woff = pk.woff;
    in.K = D.K;
    in.Nm = D.Nm;
    in.Khat = D.Khat;
    in.rinv = rinv;
    if (rinv) rinv += D.n;
    in.C = (plain || !w.Cacc.p) ? nullptr : (uint32_t*)w.Cacc.p + cacc;
    cacc += (uint64_t)(c->M + 1) * D.n * D.n;
    in.seq0 = D.seq0;
    in.win0 = D.win0;
    in.n = (uint32_t)D.n;
    in.tile0 = ftile;
    D.tile0 = ftile;
    const uint32_t nt = (uint32_t)((D.n + 31) / 32);
    ftile += nt * nt;
    memcpy(t.buf.data() + p.o_info + d * sizeof(DsInfo), &in, sizeof in);
  }
  return ftile;
}

// Device memory for a Gram plan; then serialise and upload the tables.
int plan_memory_and_tables(gakco_ctx* c, Work& w, Plan& p, bool plain) {
  const uint64_t G = p.gtot;
  const uint64_t nm = c->masks.size();
  int rc;
  ENSURE(fullkey, G * 8);
  ENSURE(wid, G * 4);
  const uint64_t pool = plain ? G : nm * G;
  ENSURE(ewin, pool * 4);
  ENSURE(eseq, pool * 4 + 16);  // 16-byte vector reads may run past the last entry
  ENSURE(efe, pool * 4);
  if ((rc = ensure_sort_buffers(c, w, p)) != GAKCO_OK) return rc;
  uint64_t nsum = 0;
  for (auto& D : p.ds) nsum += (uint64_t)D.n;
  ENSURE(rinv, nsum * 8);
  if (plain) ENSURE(Cplain, (uint64_t)(c->M + 1) * p.nmax * p.nmax * 4);
  uint64_t csum = 0;
  for (auto& D : p.ds) csum += (uint64_t)(c->M + 1) * D.n * D.n;
  p.c_elems = plain ? 0 : csum;
  if (!plain) ENSURE(Cacc, csum * 4);
  if (!p.dprobs.empty()) {
    ENSURE(Adense, p.dense_abytes);
    ENSURE(dmaxc, (p.ds.size() * (c->M + 1) + 1) * 4);  // per (dataset, level), + the overflow counter
    ENSURE(dovf, (size_t)c->dense_overflow * sizeof(DenseOvf));
  }
  if (!p.heavy.empty()) {
    ENSURE(Aheavy, p.heavy_abytes);
    ENSURE(hctr, (2 * p.heavy.size() + 1) * 4);  // columns and largest count per problem, list length
    ENSURE(hlist, p.heavy_list * sizeof(HeavyItem));
  }
  Tables t;
  add_common_tables(c, p, t);
  if ((rc = ensure(c, w, w.tables, t.buf.size(), "tables")) != GAKCO_OK) return rc;
  p.ftiles = fill_records(c, w, p, t, plain);
  if (!p.dprobs.empty() && (rc = fill_dense(c, w, p, t)) != GAKCO_OK) return rc;
  return upload_tables(c, w, t);
}

AccParams acc_params(gakco_ctx* c, Work& w, const Plan& p, uint32_t* counter) {
  uint8_t* base = (uint8_t*)w.tables.p;
  AccParams a{};
  a.ds = (const DsInfo*)(base + p.o_info);
  a.items = (const uint32_t*)(base + p.o_items);
  a.nitems = (uint32_t)(p.items.size() / kItemWords);
  a.counter = counter;
  a.M = (uint32_t)c->M;
  a.gtot = p.gtot;
  a.ewin = (const uint32_t*)w.ewin.p;
  a.eseq = (const uint32_t*)w.eseq.p;
  a.efe = (const uint32_t*)w.efe.p;
  a.ncols = p.ncols;
  a.status = (uint32_t*)w.status.p;
  a.work = (unsigned long long*)((uint8_t*)w.status.p + 64);
  memcpy(a.h, c->h, sizeof a.h);
  memcpy(a.ie, c->ie, sizeof a.ie);
  return a;
}

enum class Tail { kGram, kFit, kCross };

// Sort and run-length pass over one chunk, then the entry finalisation of
// the given kind.
void enqueue_chunk(gakco_ctx* c, Work& w, const Plan& p, const Chunk& ch, Tail tail,
                   const TrainIndex* tr = nullptr, const CrossOut* xo = nullptr) {
  uint8_t* base = (uint8_t*)w.tables.p;
  const SegDesc* segs = (const SegDesc*)(base + p.o_segs) + ch.seg_first;
  const uint32_t* tseg = (const uint32_t*)(base + p.o_tiles) + ch.tile_first;
  const MaskDesc* masks = (const MaskDesc*)(base + p.o_masks);
  const uint32_t* levels = (const uint32_t*)(base + p.o_level);
  void* kbuf[2] = {w.keyA.p, w.keyB.p};
  uint32_t* vbuf[2] = {(uint32_t*)w.valA.p, (uint32_t*)w.valB.p};
  void* kin = kbuf[1];  // the first pass extracts the masked keys here
  const uint32_t* vin = (const uint32_t*)w.wid.p;  // first-pass payload: window ids
  int cur = 0;
  bool os = use_onesweep(c) && ch.passes.size() <= (size_t)kOsMaxPasses;
  for (const auto& ps : ch.passes) os = os && ps.second <= 8;
  if (os) {
    const int np = (int)ch.passes.size();
    OsPasses ps{};
    ps.np = np;
    for (int q = 0; q < np; ++q) {
      ps.shift[q] = ch.passes[q].first;
      ps.bits[q] = ch.passes[q].second;
    }
    // Status words are told apart by their pass's epoch (1..65535); they
    // are cleared at the plan's first chunk, whenever the epochs wrap and
    // for every chunk of the plain engine (which visits chunks out of plan
    // order).
    constexpr uint64_t kEpochs = 65535;
    const bool wrap = ch.pass0 > 0 && (ch.pass0 + np - 1) / kEpochs != (ch.pass0 - 1) / kEpochs;
    if (ch.pass0 == 0 || wrap || c->engine == 1) {
      cudaMemsetAsync(w.osst.p, 0, (size_t)p.max_chunk_tiles * kOsRadix * 8, w.cs);
      if (ch.pass0 == 0 || c->engine == 1) cudaMemsetAsync(w.osctr.p, 0, (size_t)(p.total_passes + 1) * 4, w.cs);
    }
    cudaMemsetAsync(w.oscnt.p, 0, (size_t)ch.nseg * np * kOsRadix * 4, w.cs);
    {
      Bracket b(c, w, "sort_pass", 2);
      launch_os_hist(ch.wide, segs, ch.nseg, tseg, ch.ntiles, masks, (const uint64_t*)w.fullkey.p, kin,
                     (uint32_t*)w.oscnt.p, ps, w.cs);
    }
    for (int q = 0; q < np; ++q) {
      Bracket b(c, w, "sort_pass", 1);
      const uint64_t pass = ch.pass0 + (uint64_t)q;
      launch_os_scatter(ch.wide, q == 0, segs, tseg, ch.ntiles, kin, vin, kbuf[cur], vbuf[cur],
                        (const uint32_t*)w.oscnt.p, np, q, ch.passes[q].first, ch.passes[q].second,
                        (uint64_t*)w.osst.p, (uint32_t*)w.osctr.p + pass, (uint32_t)(pass % kEpochs + 1),
                        (uint32_t*)w.status.p, w.cs);
      kin = kbuf[cur];
      vin = vbuf[cur];
      cur ^= 1;
    }
  } else {
    for (size_t q = 0; q < ch.passes.size(); ++q) {
      Bracket b(c, w, "sort_pass", 4);
      launch_sort_pass(ch.wide, q == 0, segs, ch.nseg, tseg, ch.ntiles, masks,
                       (const uint64_t*)w.fullkey.p, kin, vin, kbuf[cur], vbuf[cur],
                       (uint32_t*)w.hist.p, (uint32_t*)w.dtot.p, ch.passes[q].first, ch.passes[q].second,
                       w.cs);
      kin = kbuf[cur];
      vin = vbuf[cur];
      cur ^= 1;
    }
  }
  if (tail == Tail::kGram) {
    {
      Bracket b(c, w, "run_length", 4);
      launch_rle_gram(ch.wide, segs, ch.nseg, tseg, ch.ntiles, kin, vin, (const DsPack*)(base + p.o_pack),
                      (uint32_t*)w.tcnt.p, (uint32_t*)w.segtot.p, (uint32_t*)w.trec.p, (uint32_t*)w.ewin.p,
                      (uint32_t*)w.eseq.p, (uint32_t*)w.efe.p,
                      (unsigned long long*)((uint8_t*)w.status.p + 64) + 3, c->rle_items, w.cs);
    }
    if (!p.heavy.empty() && p.heavy_level[ch.level]) {
      Bracket b(c, w, "heavy_mark", 1);
      launch_heavy_mark(segs, tseg, ch.ntiles, (const uint32_t*)w.segtot.p, levels,
                        (const uint32_t*)(base + p.o_hmap), (uint32_t)(c->M + 1),
                        (const HeavyProb*)(base + p.o_hprobs), (const uint32_t*)w.eseq.p,
                        (const uint32_t*)w.efe.p, (HeavyItem*)w.hlist.p,
                        (uint32_t*)w.hctr.p + 2 * p.heavy.size(), w.cs);
    }
    return;
  }
  Bracket b(c, w, "run_length", tail == Tail::kFit ? 5 : 4);
  launch_rle_head(ch.wide, segs, ch.nseg, tseg, ch.ntiles, kin, vin, (const DsPack*)(base + p.o_pack),
                  (uint32_t*)w.tcnt.p, (uint32_t*)w.segtot.p, (uint32_t*)w.estart.p,
                  (uint32_t*)w.etseq.p, (uint32_t*)w.efid.p, (uint32_t*)w.fstart.p,
                  (uint32_t*)w.ewin.p, w.cs);
  if (tail == Tail::kCross) {
    launch_cross_final(ch.wide, segs, tseg, ch.ntiles, (const uint32_t*)w.segtot.p, kin,
                       (const uint32_t*)w.estart.p, (const uint32_t*)w.etseq.p, levels, *tr, *xo, w.cs);
    return;
  }
  launch_rle_final(segs, tseg, ch.ntiles, (const uint32_t*)w.segtot.p, (const uint32_t*)w.estart.p,
                   (const uint32_t*)w.etseq.p, (const uint32_t*)w.efid.p, (const uint32_t*)w.fstart.p,
                   (uint32_t*)w.eseq.p, (uint32_t*)w.efe.p, w.cs);
  if (tail == Tail::kFit)
    launch_train_index(ch.wide, segs, tseg, ch.ntiles, (const uint32_t*)w.segtot.p, kin,
                       (const uint32_t*)w.estart.p, (const uint32_t*)w.fstart.p,
                       (const uint32_t*)w.eseq.p, levels, *tr, w.cs);
}

// Everything of a Gram call after the table upload, on w.cs.
int enqueue_gram(gakco_ctx* c, Work& w, const Plan& p, bool plain) {
  uint8_t* base = (uint8_t*)w.tables.p;
  uint32_t* status = (uint32_t*)w.status.p;
  cudaMemsetAsync(status, 0, 128, w.cs);
  {
    Bracket b(c, w, "pack", 1);
    launch_pack((const DsPack*)(base + p.o_pack), (uint32_t)p.ds.size(), p.nseq, c->g, c->bits,
                c->sigma, (uint64_t*)w.fullkey.p, (uint32_t*)w.wid.p, status, w.cs);
  }
  AccParams a = acc_params(c, w, p, status + 8);
  if (!plain) {
    if (p.c_elems) cudaMemsetAsync(w.Cacc.p, 0, p.c_elems * 4, w.cs);
    const uint32_t nh = (uint32_t)p.heavy.size();
    if (nh) cudaMemsetAsync(w.hctr.p, 0, (2 * (size_t)nh + 1) * 4, w.cs);
    // Dense levels (tensor cores) and sparse levels (sort, run-length,
    // on-chip accumulation) write disjoint levels of C and share only
    // read-only inputs, so they run as two branches (except when profiling,
    // where every launch is timed on one stream).  The heavy features'
    // contraction joins the dense branch once the sparse branch has built
    // its matrices; it and the accumulation add disjoint pairs of features
    // into the same C_m with atomics.
    const bool fork = c->overlap && !c->profile && (!p.dwaves.empty() || nh > 0);
    cudaStream_t ds = w.cs;
    if (fork) {
      cudaEventRecord(w.ev_fork, w.cs);
      cudaStreamWaitEvent(w.cs2, w.ev_fork, 0);
      ds = w.cs2;
    }
    if (!p.dwaves.empty()) {
      // Dense levels: A = counts per (sequence, mask, key), C_m += A A^T.
      const DenseProb* probs = (const DenseProb*)(base + p.o_dprobs);
      const uint32_t* tiles = (const uint32_t*)(base + p.o_dtiles);
      const size_t nmax_words = p.ds.size() * (size_t)(c->M + 1);
      uint32_t* ovf_n = (uint32_t*)w.dmaxc.p + nmax_words;
      const uint32_t cap = (uint32_t)c->dense_overflow;
      const int gemm_ctas = c->dense_sms > 0 ? std::min(c->dense_sms, c->nsm) : c->nsm;
      cudaMemsetAsync(w.dmaxc.p, 0, nmax_words * 4, ds);
      // Optionally (one wave, two branches) the GEMM waits for the sparse
      // levels' sort and run-length passes, so that it runs beside the
      // accumulation rather than beside them.
      const bool late = c->dense_late && fork && p.dwaves.size() == 1 && !p.chunks.empty();
      for (const DenseWave& wv : p.dwaves) {
        cudaMemsetAsync(ovf_n, 0, 4, ds);
        {
          Bracket b(c, w, "dense_scatter", 1);
          launch_dense_scatter(probs + wv.p0, wv.np, wv.p0, wv.rows, (const DsPack*)(base + p.o_pack),
                               (const MaskDesc*)(base + p.o_masks), (const uint64_t*)w.fullkey.p,
                               (uint32_t)(c->g * c->bits), ovf_n, (DenseOvf*)w.dovf.p, cap, ds);
        }
        if (late) {
          for (const Chunk& ch : p.chunks) enqueue_chunk(c, w, p, ch, Tail::kGram);
          cudaEventRecord(w.ev_sparse, w.cs);
          cudaStreamWaitEvent(ds, w.ev_sparse, 0);
        }
        {
          Bracket b(c, w, "dense_gemm", 1);
          launch_dense_gemm(probs, tiles + kDenseTileWords * (size_t)wv.t0, wv.nt, gemm_ctas,
                            (uint32_t)c->dense_round_sum, (long long)c->dense_wait_cycles, status, ds);
        }
        Bracket b(c, w, "dense_fix", 1);
        launch_dense_fix(probs, ovf_n, (const DenseOvf*)w.dovf.p, cap, status, ds);
      }
      if (!late)
        for (const Chunk& ch : p.chunks) enqueue_chunk(c, w, p, ch, Tail::kGram);
    } else {
      for (const Chunk& ch : p.chunks) enqueue_chunk(c, w, p, ch, Tail::kGram);
    }
    if (nh) {
      const HeavyProb* hp = (const HeavyProb*)(base + p.o_hprobs);
      const uint32_t* nitems = (const uint32_t*)w.hctr.p + 2 * nh;
      {
        Bracket b(c, w, "heavy_prep", 2);
        launch_heavy_zero(hp, nh, p.heavy_rows, (DenseProb*)(base + p.o_dprobs),
                          (unsigned long long*)((uint8_t*)w.status.p + 96), w.cs);
        launch_heavy_scatter(hp, (const HeavyItem*)w.hlist.p, nitems, (uint32_t*)w.eseq.p, (uint32_t*)w.efe.p,
                             c->nsm, w.cs);
      }
      cudaStream_t hs = w.cs;
      if (fork) {
        cudaEventRecord(w.ev_heavy, w.cs);
        cudaStreamWaitEvent(w.cs2, w.ev_heavy, 0);
        hs = w.cs2;
      }
      Bracket b(c, w, "heavy_gemm", 1);
      const int gemm_ctas = c->dense_sms > 0 ? std::min(c->dense_sms, c->nsm) : c->nsm;
      launch_dense_gemm((const DenseProb*)(base + p.o_dprobs),
                        (const uint32_t*)(base + p.o_dtiles) + kDenseTileWords * (size_t)p.heavy_t0, p.heavy_nt,
                        gemm_ctas, (uint32_t)c->dense_round_sum, (long long)c->dense_wait_cycles, status, hs);
    }
    if (fork) cudaEventRecord(w.ev_join, w.cs2);
    {
      Bracket b(c, w, "accumulate", 1);
      launch_accum(a, c->accum_threads, c->accum_variant, p.acc_blocks, p.acc_smem, w.cs);
    }
    if (fork) cudaStreamWaitEvent(w.cs, w.ev_join, 0);
    if (p.partial_C) {
      // A partial Gram: this slice's C_0..C_M (upper triangles) go to the
      // caller, who sums the slices and finishes with gakco_combine_device.
      if (p.c_elems) cudaMemcpyAsync(p.partial_C, w.Cacc.p, p.c_elems * 4, cudaMemcpyDeviceToDevice, w.cs);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return wcuda(w, e, "kernel launch");
      return GAKCO_OK;
    }
    {
      Bracket b(c, w, "diag", 1);
      launch_diag((const DsInfo*)(base + p.o_info), (uint32_t)p.ds.size(), p.nseq, a, w.cs);
    }
    Bracket b(c, w, "combine", 1);
    launch_combine((const DsInfo*)(base + p.o_info), (uint32_t)p.ds.size(), p.ftiles, a, p.want_nm,
                   p.want_khat, w.cs);
  } else {
    const DsInfo* infos = (const DsInfo*)(base + p.o_info);
    // Chunks are one segment each and ordered by level, then mask, then
    // dataset; handle one dataset at a time so C_m fits one buffer.
    for (size_t d = 0; d < p.ds.size(); ++d) {
      const DsHost& D = p.ds[d];
      if (D.n == 0) continue;
      const uint64_t nn = (uint64_t)D.n * D.n;
      cudaMemsetAsync(w.Cplain.p, 0, (size_t)(c->M + 1) * nn * 4, w.cs);
      for (const Chunk& ch : p.chunks) {
        if (p.seg_ds[ch.seg_first] != d) continue;
        const SegDesc& s = p.segs[ch.seg_first];
        enqueue_chunk(c, w, p, ch, Tail::kGram);
        Bracket b(c, w, "pairs_global", 1);
        launch_pairs_global((const uint32_t*)w.segtot.p, (const uint32_t*)w.eseq.p + s.pool,
                            (const uint32_t*)w.efe.p + s.pool, s.G,
                            (uint32_t*)w.Cplain.p + (uint64_t)ch.level * nn, (uint32_t)D.n, status,
                            w.cs);
      }
      Bracket b(c, w, "ie_combine", 1);
      launch_ie_combine(infos + d, (const uint32_t*)w.Cplain.p, (uint32_t)D.n, a, w.cs);
    }
    Bracket b(c, w, "finish", 1);
    launch_finish(infos, (uint32_t)p.ds.size(), p.ftiles, (uint32_t)c->M, p.want_nm, p.want_khat, w.cs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wcuda(w, e, "kernel launch");
  return GAKCO_OK;
}

uint64_t plan_key(gakco_ctx* c, const Plan& p, bool plain) {
  uint64_t h = 1469598103934665603ull;
  int64_t o[16] = {plain,           c->radix_bits, c->chunk_elems, c->accum_threads,  c->smem_cols,
                   (int64_t)p.ds.size(), c->group_bytes, c->dense,    c->dense_bytes, c->dense_overflow,
                   c->dense_run_cols, p.first_level, c->overlap, c->dense_sms, c->heavy, c->heavy_bytes};
  h = fnv1a(h, o, sizeof o);
  for (const DsHost& D : p.ds) {
    const void* ptrs[4] = {D.codes, D.K, D.Khat, D.Nm};
    h = fnv1a(h, ptrs, sizeof ptrs);
    h = fnv1a(h, &D.n, sizeof D.n);
    if (D.n > 0) h = fnv1a(h, D.off, (D.n + 1) * 8);
  }
  return h;
}

// Device status word -> error code (after the status has reached h_status).
int check_status(gakco_ctx* c, Work& w) {
  const uint32_t st = ((const uint32_t*)w.h_status)[0];
  const unsigned long long* wk = (const unsigned long long*)((const uint8_t*)w.h_status + 64);
  w.pairs = (double)wk[0];
  w.entries = (double)wk[1];
  w.windows = (double)wk[2];
  w.rle_entries = (double)wk[3];
  w.heavy_cols = (double)wk[4];
  w.heavy_flops = (double)wk[5];
  if (st & kErrBadCode) return wfail(w, GAKCO_E_INVALID, "input holds a symbol >= sigma (%d)", c->sigma);
  // A full overflow list leaves the dense levels uncorrected (which later
  // checks may flag too): the caller reruns the call with every level
  // sparse, so this comes first.
  if (st & kErrDenseOverflow) {
    w.dense_overflow = true;
    return wfail(w, GAKCO_E_INTERNAL, "dense overflow list full");
  }
  if (st & kErrKneCM) return wfail(w, GAKCO_E_INTERNAL, "internal check failed: sum h_m N_m != C_M");
  if (st & kErrBadEntry) return wfail(w, GAKCO_E_INTERNAL, "internal check failed: entry out of range");
  if (st & kErrTimeout) return wfail(w, GAKCO_E_TIMEOUT, "a bounded wait in the dense GEMM ran out");
  if (st) return wfail(w, GAKCO_E_INTERNAL, "device status 0x%x", st);
  return GAKCO_OK;
}

int sync_and_check(gakco_ctx* c, Work& w) {
  w.dense_overflow = false;
  cudaError_t e = cudaMemcpyAsync(w.h_status, w.status.p, 128, cudaMemcpyDeviceToHost, w.cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "engine run");
  if (c->profile && &w == &c->main) {
    c->timings.clear();
    for (const Timed& t : c->timed) {
      float ms = 0;
      cudaEventElapsedTime(&ms, t.a, t.b);
      bool found = false;
      for (auto& kv : c->timings)
        if (kv.first == t.name) {
          kv.second.first += ms;
          kv.second.second += 1;
          found = true;
        }
      if (!found) c->timings.push_back({t.name, {ms, 1}});
    }
  }
  return check_status(c, w);
}

int run_gram_once(gakco_ctx* c, Plan& p, cudaStream_t user);

// The batched / plain Gram engine on device buffers, on the context's Work.
// When a dense level met more counts above 16 than its overflow list holds,
// the call is run again with every level on the sparse route, so results
// stay exact.
int run_gram(gakco_ctx* c, Plan& p, cudaStream_t user) {
  c->main.dense_overflow = false;
  Plan q;  // the validated datasets alone, for a second run
  q.ds = p.ds;
  q.gtot = p.gtot;
  q.nseq = p.nseq;
  q.nmax = p.nmax;
  q.want_nm = p.want_nm;
  q.want_khat = p.want_khat;
  q.mask_lo = p.mask_lo;
  q.mask_hi = p.mask_hi;
  q.partial_C = p.partial_C;
  int rc = run_gram_once(c, p, user);
  if (rc != GAKCO_OK && c->main.dense_overflow && c->dense != 0) {
    const int saved = c->dense;
    c->dense = 0;
    drop_graph(c);
    rc = run_gram_once(c, q, user);
    c->dense = saved;
    drop_graph(c);
  }
  return rc;
}

int run_gram_once(gakco_ctx* c, Plan& p, cudaStream_t user) {
  Work& w = c->main;
  const bool plain = c->engine == 1;
  w.launches = 0;
  c->timed.clear();
  c->ev_used = 0;
  c->last_replay = 0;
  c->last_mask_passes = 0;
  p.first_level = (c->kernel_only && !p.want_nm && !plain && !p.partial_C) ? c->M : 0;
  const int64_t masks_run =
      std::max<int64_t>(0, std::min<int64_t>((int64_t)c->masks.size(), (int64_t)p.mask_hi) -
                               std::max<int64_t>((int64_t)level_firsts(c)[p.first_level], (int64_t)p.mask_lo));
  for (const DsHost& D : p.ds)
    if (D.G > 0) c->last_mask_passes += masks_run;
  if (p.ds.empty()) {
    c->last_launches = 0;
    return GAKCO_OK;
  }
  cudaError_t e = cudaEventRecord(c->ev_in, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w.cs, c->ev_in, 0);
  if (e != cudaSuccess) return wcuda(w, e, "stream ordering");

  const bool graph = c->use_graph && !c->profile && !plain && !p.partial_C;
  const uint64_t key = graph ? plan_key(c, p, plain) : 0;
  int rc;
  if (graph && c->gexec && key == c->gkey) {
    // Same plan as the cached graph: tables and buffers are unchanged.
    e = cudaGraphLaunch(c->gexec, w.cs);
    if (e != cudaSuccess) return wcuda(w, e, "graph launch");
    w.launches = c->last_launches;
    c->last_replay = 1;
  } else {
    drop_graph(c);
    plan_dense(c, p, plain);
    c->plan_dense_probs = (double)p.dprobs.size();
    plan_heavy(c, p, plain);
    plan_chunks(c, p, plain);
    c->plan_dense_flops = p.dense_flops;
    c->plan_dense_issued = p.dense_issued;
    c->plan_dense_bytes = p.dense_bytes;
    c->plan_sort_bytes = p.sort_bytes;
    c->plan_rle_bytes = p.rle_bytes;
    plan_io_bytes(c, p);
    c->plan_pack_bytes = p.pack_bytes;
    c->plan_combine_bytes = p.combine_bytes;
    plan_items(c, p);
    if (!plain) {
      const int nb = accum_blocks_per_sm(c->accum_threads, c->accum_variant, p.acc_smem);
      if (nb <= 0)
        return wfail(w, GAKCO_E_CUDA, "accumulation kernel does not fit (%zu B shared)", p.acc_smem);
      p.acc_blocks = nb * c->nsm;
    }
    if ((rc = plan_memory_and_tables(c, w, p, plain)) != GAKCO_OK) return rc;
    if (graph) {
      cudaGraph_t gr = nullptr;
      e = cudaStreamBeginCapture(w.cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return wcuda(w, e, "begin capture");
      rc = enqueue_gram(c, w, p, plain);
      e = cudaStreamEndCapture(w.cs, &gr);
      if (rc != GAKCO_OK) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return wcuda(w, e, "end capture");
      e = cudaGraphInstantiate(&c->gexec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        c->gexec = nullptr;
        return wcuda(w, e, "graph instantiate");
      }
      c->gkey = key;
      e = cudaGraphLaunch(c->gexec, w.cs);
      if (e != cudaSuccess) return wcuda(w, e, "graph launch");
    } else {
      if ((rc = enqueue_gram(c, w, p, plain)) != GAKCO_OK) return rc;
    }
  }
  c->last_launches = w.launches;
  rc = sync_and_check(c, w);
  c->last_pairs = w.pairs;
  c->last_entries = w.entries;
  c->last_windows = w.windows;
  c->last_heavy_cols = w.heavy_cols;
  c->last_heavy_flops = w.heavy_flops;
  c->last_rle_entries = w.rle_entries;
  e = cudaEventRecord(c->ev_out, w.cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, c->ev_out, 0);
  if (e != cudaSuccess && rc == GAKCO_OK) rc = wcuda(w, e, "stream ordering");
  return rc;
}

int gram_host(gakco_ctx* c, int32_t nd, const uint8_t* const* codes, const int64_t* const* off,
              const int32_t* n, int32_t* const* K, double* const* Khat, int32_t* const* Nm) {
  Work& w = c->main;
  Plan p;
  int rc = plan_datasets(c, w, p, nd, codes, off, n, K, Khat, Nm, false);
  if (rc != GAKCO_OK) return rc;
  // Stage codes and outputs in the context's device buffers.
  uint64_t cbytes = 0, kel = 0, nmel = 0;
  bool want_khat = false, want_nm = false;
  std::vector<uint64_t> coff(nd), koff(nd), nmoff(nd);
  for (int32_t d = 0; d < nd; ++d) {
    const DsHost& D = p.ds[d];
    coff[d] = cbytes;
    if (D.n > 0) cbytes += (uint64_t)(D.off[D.n]);
    cbytes = align_up(cbytes, 16);
    koff[d] = kel;
    kel += (uint64_t)D.n * D.n;
    nmoff[d] = nmel;
    if (D.Nm) nmel += (uint64_t)(c->M + 1) * D.n * D.n;
    want_khat |= D.Khat != nullptr;
    want_nm |= D.Nm != nullptr;
  }
  ENSURE(codes, cbytes + 16);
  ENSURE(outK, kel * 4 + 16);
  if (want_khat) ENSURE(outKhat, kel * 8 + 16);
  if (want_nm) ENSURE(outNm, nmel * 4 + 16);
  cudaError_t e = cudaSuccess;
  for (int32_t d = 0; d < nd && e == cudaSuccess; ++d) {
    DsHost& D = p.ds[d];
    const uint8_t* dc = (const uint8_t*)w.codes.p + coff[d];
    if (D.n > 0 && D.off[D.n] > 0)
      e = cudaMemcpyAsync((void*)dc, D.codes, (size_t)D.off[D.n], cudaMemcpyHostToDevice, w.cs);
    D.codes = dc;
    D.K = (int32_t*)w.outK.p + koff[d];
    D.Khat = D.Khat ? (double*)w.outKhat.p + koff[d] : nullptr;
    D.Nm = D.Nm ? (int32_t*)w.outNm.p + nmoff[d] : nullptr;
  }
  if (e != cudaSuccess) return wcuda(w, e, "copy codes to device");
  std::vector<Xfer> xs;
  for (int32_t d = 0; d < nd; ++d) {
    const DsHost& D = p.ds[d];
    const size_t nn = (size_t)D.n * D.n;
    if (!nn) continue;
    if (K && K[d]) xs.push_back({K[d], D.K, nn * 4});
    if (Khat && Khat[d]) xs.push_back({Khat[d], D.Khat, nn * 8});
    if (Nm && Nm[d]) xs.push_back({Nm[d], D.Nm, (size_t)(c->M + 1) * nn * 4});
  }
  const bool direct = direct_copies(c);
  PageTouch touch(direct, xs);
  rc = run_gram(c, p, w.cs);
  touch.wait();
  if (rc != GAKCO_OK) return rc;
  return copy_to_host(w, xs, direct);
}

// --------------------------------------------------------- training index --

TrainIndex train_index(const Train& T) {
  TrainIndex tr{};
  tr.ukey = (uint64_t*)T.ukey.p;
  tr.ufirst = (uint32_t*)T.ufirst.p;
  tr.eseq = (uint32_t*)T.eseq.p;
  tr.nfeat = (uint32_t*)T.nfeat.p;
  tr.diagC = (uint32_t*)T.diagC.p;
  tr.rinv = (double*)T.rinv.p;
  tr.stride = T.G + 1;
  tr.n = (uint32_t)T.n;
  return tr;
}

TrainIndex train_index(gakco_ctx* c) { return train_index(c->train); }

CrossParams cross_params(gakco_ctx* c, Work& w) {
  CrossParams x{};
  x.tr = train_index(c);
  x.M = (uint32_t)c->M;
  x.status = (uint32_t*)w.status.p;
  memcpy(x.h, c->h, sizeof x.h);
  memcpy(x.ie, c->ie, sizeof x.ie);
  return x;
}

// Build the resident index of a training set (device codes, host offsets).
// The per-mask training index of a set of sequences (device codes, host
// offsets) into T: sort and count every mask, keep the features, their
// first entries and the entries, and the diagonal and norms.  Enqueued on
// the main Work's stream; does not wait.
int build_index(gakco_ctx* c, Train& T, const uint8_t* d_codes, const int64_t* off, int32_t n) {
  Work& w = c->main;
  // The cached Gram graph points into w's tables and buffers, which this
  // call rewrites and may reallocate.
  drop_graph(c);
  Plan p;
  int rc = plan_datasets(c, w, p, 1, &d_codes, &off, &n, nullptr, nullptr, nullptr, false);
  if (rc != GAKCO_OK) return rc;
  const DsHost& D = p.ds[0];
  plan_chunks(c, p, false);
  const uint64_t G = p.gtot, nm = c->masks.size(), stride = G + 1;
  const uint64_t n1 = (uint64_t)std::max(n, 1);
  ENSURE(fullkey, G * 8);
  ENSURE(wid, G * 4);
  ENSURE(ewin, nm * G * 4);
  ENSURE(eseq, nm * G * 4);
  ENSURE(efe, nm * G * 4);
  if ((rc = ensure_sort_buffers(c, w, p)) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, T.ukey, nm * stride * 8, "train keys")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, T.ufirst, nm * stride * 4, "train features")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, T.eseq, nm * stride * 4, "train entries")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, T.nfeat, nm * 4, "train feature counts")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, T.diagC, (uint64_t)(c->M + 1) * n1 * 4, "train diagonal")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, T.rinv, n1 * 8, "train norms")) != GAKCO_OK) return rc;
  T.n = n;
  T.G = G;
  T.woff = D.woff;
  Tables t;
  add_common_tables(c, p, t);
  if ((rc = ensure(c, w, w.tables, t.buf.size(), "tables")) != GAKCO_OK) return rc;
  fill_records(c, w, p, t, true);
  if ((rc = upload_tables(c, w, t)) != GAKCO_OK) return rc;
  w.launches = 0;
  uint8_t* base = (uint8_t*)w.tables.p;
  uint32_t* status = (uint32_t*)w.status.p;
  cudaMemsetAsync(status, 0, 128, w.cs);
  cudaMemsetAsync(T.diagC.p, 0, (size_t)(c->M + 1) * n1 * 4, w.cs);
  cudaMemsetAsync(T.nfeat.p, 0, nm * 4, w.cs);
  cudaMemsetAsync(T.ufirst.p, 0, nm * stride * 4, w.cs);
  launch_pack((const DsPack*)(base + p.o_pack), 1, p.nseq, c->g, c->bits, c->sigma,
              (uint64_t*)w.fullkey.p, (uint32_t*)w.wid.p, status, w.cs);
  const TrainIndex tr = train_index(T);
  for (const Chunk& ch : p.chunks) enqueue_chunk(c, w, p, ch, Tail::kFit, &tr);
  CrossParams x = cross_params(c, w);
  launch_vec_diag(tr.diagC, (uint32_t)n, x, tr.rinv, w.cs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wcuda(w, e, "kernel launch");
  return GAKCO_OK;
}

int fit(gakco_ctx* c, const uint8_t* d_codes, const int64_t* off, int32_t n) {
  Work& w = c->main;
  Train& T = c->train;
  T.ok = false;
  T.svm_ok = false;  // coefficients belong to the previous training set
  int rc = build_index(c, T, d_codes, off, n);
  if (rc != GAKCO_OK) return rc;
  cudaError_t e = cudaSuccess;
  // Keep the training codes: adding sequences appends to them.
  const uint64_t cbytes = n > 0 ? (uint64_t)off[n] : 0;
  if ((rc = ensure(c, w, T.tcodes, cbytes + 16, "training codes")) != GAKCO_OK) return rc;
  if (cbytes && (e = cudaMemcpyAsync(T.tcodes.p, d_codes, cbytes, cudaMemcpyDeviceToDevice, w.cs)) != cudaSuccess)
    return wcuda(w, e, "keep training codes");
  T.toff.assign(off, off + n + 1);
  if (n == 0) T.toff.assign(1, 0);
  if ((rc = sync_and_check(c, w)) != GAKCO_OK) return rc;
  T.ok = true;
  return GAKCO_OK;
}

int cross_host(gakco_ctx* c, const uint8_t* codes, const int64_t* off, int32_t nt, int32_t* K,
               double* Khat, double* F = nullptr);

// Adds nb sequences (host buffers) to the fitted set and returns the new
// rows of the union's Gram matrix (old sequences first): against the old
// sequences they are the cross kernel, among themselves the Gram kernel of
// the new block.  Khat follows the Gram engine exactly: r = 1 / sqrt(K(x, x))
// (the resident index keeps the old ones), (K * r_a) * r_b with a the
// smaller index, 1 on a nonzero diagonal.  The fitted set becomes the
// union: the new sequences' index is built and merged into the resident one
// (launch_index_merge), which leaves it identical to a fit of the union.
int extend(gakco_ctx* c, const uint8_t* codes, const int64_t* off, int32_t nb, int32_t* Krows,
           double* Khat) {
  Work& w = c->main;
  Train& T = c->train;
  int rc;
  if (!T.ok) return wfail(w, GAKCO_E_INVALID, "no training set: call gakco_fit first");
  const int32_t n = T.n;
  if (nb < 0 || (nb > 0 && !off)) return wfail(w, GAKCO_E_INVALID, "bad new sequences");
  if ((int64_t)n + nb > 65535) return wfail(w, GAKCO_E_INVALID, "n + nb = %d above 65535", n + nb);
  if (nb > 0 && !Krows) return wfail(w, GAKCO_E_INVALID, "null kernel buffer");
  const size_t N = (size_t)n + nb;
  std::vector<int32_t> kbt((size_t)nb * n), kbb((size_t)nb * nb);
  std::vector<double> rold(n);
  if (nb > 0 && n > 0) {
    if ((rc = cross_host(c, codes, off, nb, kbt.data(), nullptr)) != GAKCO_OK) return rc;
    cudaError_t e = cudaMemcpy(rold.data(), T.rinv.p, (size_t)n * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return wcuda(w, e, "copy training norms");
  }
  if (nb > 0) {
    int32_t* kp = kbb.data();
    if ((rc = gram_host(c, 1, &codes, &off, &nb, &kp, nullptr, nullptr)) != GAKCO_OK) return rc;
  }
  std::vector<double> rnew(nb);
  for (int32_t i = 0; i < nb; ++i) {
    const int32_t d = kbb[(size_t)i * nb + i];
    rnew[i] = d ? 1.0 / std::sqrt((double)d) : 0.0;
  }
  for (int32_t i = 0; i < nb; ++i) {
    int32_t* kr = Krows + (size_t)i * N;
    double* hr = Khat ? Khat + (size_t)i * N : nullptr;
    for (int32_t j = 0; j < n; ++j) {
      kr[j] = kbt[(size_t)i * n + j];
      if (hr) hr[j] = ((double)kr[j] * rold[j]) * rnew[i];
    }
    for (int32_t j = 0; j < nb; ++j) {
      const int32_t v = kbb[(size_t)i * nb + j];
      kr[n + j] = v;
      if (!hr) continue;
      if (j == i)
        hr[n + j] = rnew[i] > 0.0 ? 1.0 : 0.0;
      else if (j < i)
        hr[n + j] = ((double)v * rnew[j]) * rnew[i];
      else
        hr[n + j] = ((double)v * rnew[i]) * rnew[j];
    }
  }
  if (nb == 0) return GAKCO_OK;  // the fitted set is unchanged
  // The union's index: the new sequences' own index, merged per mask into
  // the resident one (their ids follow the old ones), then swapped in.
  const uint64_t base = (uint64_t)T.toff.back();
  const uint64_t newbytes = (uint64_t)off[nb];
  if ((rc = ensure(c, w, w.codes, newbytes + 16, "codes")) != GAKCO_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(w.codes.p, codes, newbytes, cudaMemcpyHostToDevice, w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "upload the new codes");
  Train& B = c->train_add;
  if ((rc = build_index(c, B, (const uint8_t*)w.codes.p, off, nb)) != GAKCO_OK) return rc;
  Train& U = c->train_merged;
  const uint64_t nm = c->masks.size(), L = (uint64_t)(c->M + 1);
  const uint64_t GU = T.G + B.G, su = GU + 1;
  if ((rc = ensure(c, w, U.ukey, nm * su * 8, "merged keys")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, U.ufirst, nm * su * 4, "merged features")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, U.eseq, nm * su * 4, "merged entries")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, U.nfeat, nm * 4, "merged feature counts")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, U.diagC, L * N * 4, "merged diagonal")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, U.rinv, N * 8, "merged norms")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, U.tcodes, base + newbytes + 16, "merged codes")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, w.ea, nm * (B.G + 1) * 4, "merge ranks")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, w, w.eb, nm * (B.G + 1) * 4, "merge flags")) != GAKCO_OK) return rc;
  U.n = (int32_t)N;
  U.G = GU;
  launch_index_merge(train_index(T), train_index(B), train_index(U), (uint32_t)nm, (uint32_t*)w.ea.p,
                     (uint32_t*)w.eb.p, (uint32_t)n, w.cs);
  if (n > 0) {
    e = cudaMemcpy2DAsync(U.diagC.p, N * 4, T.diagC.p, (size_t)n * 4, (size_t)n * 4, L, cudaMemcpyDeviceToDevice, w.cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(U.rinv.p, T.rinv.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, w.cs);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync((uint32_t*)U.diagC.p + n, N * 4, B.diagC.p, (size_t)nb * 4, (size_t)nb * 4, L,
                          cudaMemcpyDeviceToDevice, w.cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync((double*)U.rinv.p + n, B.rinv.p, (size_t)nb * 8, cudaMemcpyDeviceToDevice, w.cs);
  if (e == cudaSuccess && base) e = cudaMemcpyAsync(U.tcodes.p, T.tcodes.p, base, cudaMemcpyDeviceToDevice, w.cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((uint8_t*)U.tcodes.p + base, w.codes.p, newbytes, cudaMemcpyDeviceToDevice, w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "assemble the merged index");
  T.ok = false;
  if ((rc = sync_and_check(c, w)) != GAKCO_OK) return rc;
  std::swap(T.ukey, U.ukey);
  std::swap(T.ufirst, U.ufirst);
  std::swap(T.eseq, U.eseq);
  std::swap(T.nfeat, U.nfeat);
  std::swap(T.diagC, U.diagC);
  std::swap(T.rinv, U.rinv);
  std::swap(T.tcodes, U.tcodes);
  for (int32_t x = 1; x <= nb; ++x) T.woff.push_back((uint32_t)(T.G + B.woff[x]));
  for (int32_t x = 1; x <= nb; ++x) T.toff.push_back((int64_t)base + off[x]);
  T.n = (int32_t)N;
  T.G = GU;
  T.svm_ok = false;  // coefficients belong to the previous training set
  T.ok = true;
  return GAKCO_OK;
}

// Enqueue the cross kernel of one test batch on w (device codes, host
// offsets; K / Khat device outputs of nt x n_train, dF nt SVM decision
// values, each may be null).  Does not wait.
int enqueue_cross(gakco_ctx* c, Work& w, const uint8_t* d_codes, const int64_t* off, int32_t nt,
                  int32_t* dK, double* dKhat, double* dF = nullptr) {
  Train& T = c->train;
  if (!T.ok) return wfail(w, GAKCO_E_INVALID, "no training set: call gakco_fit first");
  if (dF && !T.svm_ok) return wfail(w, GAKCO_E_INVALID, "no SVM coefficients: call gakco_set_svm first");
  // On the context's own Work the cached Gram graph points into the tables
  // and buffers this call rewrites and may reallocate (serving slots have
  // their own Work).
  if (&w == &c->main) drop_graph(c);
  uint64_t twmax = 1;
  for (size_t y = 0; y + 1 < T.woff.size(); ++y) twmax = std::max<uint64_t>(twmax, T.woff[y + 1] - T.woff[y]);
  Plan p;
  int rc = plan_datasets(c, w, p, 1, &d_codes, &off, &nt, nullptr, nullptr, nullptr, false, twmax);
  if (rc != GAKCO_OK) return rc;
  const DsHost& D = p.ds[0];
  plan_chunks(c, p, false);
  const uint64_t G = p.gtot, nm = c->masks.size();
  const uint32_t ntr = (uint32_t)T.n;
  const uint32_t ncols = smem_columns(c, ntr);
  add_items(c, p.items, 0, D.woff, (uint32_t)nt, ntr, ncols, 4.0 * (double)(T.G + 1) + 16.0 * (double)G,
            false);
  const size_t smem = 4 * ((size_t)ncols + 1);
  ENSURE(fullkey, G * 8);
  ENSURE(wid, G * 4);
  ENSURE(ewin, nm * G * 4);
  ENSURE(eseq, nm * G * 4);
  ENSURE(ea, nm * G * 4);
  ENSURE(eb, nm * G * 4);
  if ((rc = ensure_sort_buffers(c, w, p)) != GAKCO_OK) return rc;
  const uint64_t cd = (uint64_t)(c->M + 1) * std::max(nt, 1);
  const uint64_t cx = cd * std::max<uint32_t>(ntr, 1);
  ENSURE(Cd, cd * 4);
  ENSURE(Cx, cx * 4);
  ENSURE(rinv, (uint64_t)std::max(nt, 1) * 8);
  Tables t;
  add_common_tables(c, p, t);
  if ((rc = ensure(c, w, w.tables, t.buf.size(), "tables")) != GAKCO_OK) return rc;
  fill_records(c, w, p, t, true);
  if ((rc = upload_tables(c, w, t)) != GAKCO_OK) return rc;
  const int nb = cross_accum_blocks_per_sm(smem);
  if (nb <= 0) return wfail(w, GAKCO_E_CUDA, "cross accumulation does not fit (%zu B shared)", smem);
  uint8_t* base = (uint8_t*)w.tables.p;
  uint32_t* status = (uint32_t*)w.status.p;
  CrossParams x = cross_params(c, w);
  x.xo.eseq = (uint32_t*)w.eseq.p;
  x.xo.ea = (uint32_t*)w.ea.p;
  x.xo.eb = (uint32_t*)w.eb.p;
  x.xo.Cd = (uint32_t*)w.Cd.p;
  x.xo.Cx = (uint32_t*)w.Cx.p;
  x.xo.rinv = (double*)w.rinv.p;
  x.xo.nt = (uint32_t)nt;
  x.items = (const uint32_t*)(base + p.o_items);
  x.nitems = (uint32_t)(p.items.size() / kItemWords);
  x.counter = status + 8;
  x.woff = (const uint32_t*)(base + p.o_woff[0]);
  x.ewin = (const uint32_t*)w.ewin.p;
  x.gt = G;
  cudaMemsetAsync(status, 0, 128, w.cs);
  cudaMemsetAsync(w.Cd.p, 0, cd * 4, w.cs);
  cudaMemsetAsync(w.Cx.p, 0, cx * 4, w.cs);
  launch_pack((const DsPack*)(base + p.o_pack), 1, p.nseq, c->g, c->bits, c->sigma,
              (uint64_t*)w.fullkey.p, (uint32_t*)w.wid.p, status, w.cs);
  const TrainIndex tr = x.tr;
  for (const Chunk& ch : p.chunks) enqueue_chunk(c, w, p, ch, Tail::kCross, &tr, &x.xo);
  launch_cross_accum(x, nb * c->nsm, smem, w.cs);
  launch_vec_diag(x.xo.Cd, (uint32_t)nt, x, x.xo.rinv, w.cs);
  launch_cross_combine(x, dK, dKhat, w.cs);
  w.launches += 5;
  if (dF) {
    launch_svm_decision(x, (const double*)T.svm.p, T.svm_bias, T.svm_kind, dF, w.cs);
    w.launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wcuda(w, e, "kernel launch");
  return GAKCO_OK;
}

// Synchronous cross kernel on host buffers, on the context's Work (F: SVM
// decision values, nt, or null).
int cross_host(gakco_ctx* c, const uint8_t* codes, const int64_t* off, int32_t nt, int32_t* K,
               double* Khat, double* F) {
  Work& w = c->main;
  int rc;
  if (nt < 0 || nt > 65535) return wfail(w, GAKCO_E_INVALID, "nt = %d outside [0, 65535]", nt);
  if (nt > 0 && !off) return wfail(w, GAKCO_E_INVALID, "null offsets");
  if (!c->train.ok) return wfail(w, GAKCO_E_INVALID, "no training set: call gakco_fit first");
  if (nt == 0) return GAKCO_OK;
  const uint64_t cbytes = (uint64_t)off[nt];
  const uint64_t nel = (uint64_t)nt * c->train.n;
  ENSURE(codes, cbytes + 16);
  ENSURE(outK, nel * 4 + 16);
  ENSURE(outKhat, nel * 8 + 16);
  if (F) ENSURE(outF, (size_t)nt * 8);
  cudaError_t e = cudaSuccess;
  if (cbytes) e = cudaMemcpyAsync(w.codes.p, codes, cbytes, cudaMemcpyHostToDevice, w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "copy codes to device");
  std::vector<Xfer> xs;
  if (K && nel) xs.push_back({K, w.outK.p, nel * 4});
  if (Khat && nel) xs.push_back({Khat, w.outKhat.p, nel * 8});
  if (F) xs.push_back({F, w.outF.p, (size_t)nt * 8});
  const bool direct = direct_copies(c);
  PageTouch touch(direct, xs);
  if ((rc = enqueue_cross(c, w, (const uint8_t*)w.codes.p, off, nt, K ? (int32_t*)w.outK.p : nullptr,
                          Khat ? (double*)w.outKhat.p : nullptr, F ? (double*)w.outF.p : nullptr)) != GAKCO_OK)
    return rc;
  rc = sync_and_check(c, w);
  touch.wait();
  if (rc != GAKCO_OK) return rc;
  return copy_to_host(w, xs, direct);
}

// ---------------------------------------------------------------- serving --
//
// Requests are admitted into slots (a Work each: stream, device buffers,
// pinned staging).  A free slot takes the longest prefix of the queue that
// fits its limits (sequences, windows) as one micro-batch; the memory budget
// holds a batch back while other slots are busy.  Each batch runs
// asynchronously on its slot's stream and a host callback marks it done, so
// several batches overlap on the device and requests that arrive meanwhile
// are admitted as slots free up.  Results are exact integers and elementwise
// fp64, so a request's rows do not depend on the batch it ran in.

void CUDART_CB on_slot_done(void* arg) {
  // Runs on a driver thread after the slot's copies: only raise the flag;
  // the dispatcher polls it at least every 50 microseconds.
  ((Slot*)arg)->gpu_done.store(true);
}

uint64_t req_windows(const gakco_ctx* c, const Request* r) {
  uint64_t W = 0;
  for (int32_t x = 0; x < r->nt; ++x) {
    const int64_t len = r->off[x + 1] - r->off[x];
    if (len >= c->g) W += (uint64_t)(len - c->g + 1);
  }
  return W;
}

// Launch one micro-batch on a slot (no lock held).
int launch_batch(gakco_ctx* c, Slot& s) {
  Work& w = s.w;
  int rc;
  std::vector<int64_t> off(1, 0);
  size_t cbytes = 0;
  s.row0.clear();
  int32_t nt = 0;
  for (Request* r : s.batch) {
    s.row0.push_back(nt);
    for (int32_t x = 0; x < r->nt; ++x) off.push_back(off.back() + (r->off[x + 1] - r->off[x]));
    nt += r->nt;
    cbytes += (size_t)(r->off[r->nt] - r->off[0]);
  }
  s.nt = nt;
  const uint32_t ntr = (uint32_t)c->train.n;
  const size_t nel = (size_t)nt * ntr;
  bool want_f = false;
  for (Request* r : s.batch) want_f |= r->F != nullptr;
  s.k_off = align_up(cbytes, 256);
  s.kh_off = align_up(s.k_off + nel * 4, 256);
  s.f_off = align_up(s.kh_off + nel * 8, 256);
  if ((rc = ensure_pinned(w, w.h_io, w.h_io_cap, s.f_off + (size_t)nt * 8 + 256, "serve staging")) != GAKCO_OK)
    return rc;
  uint8_t* hio = (uint8_t*)w.h_io;
  size_t pos = 0;
  for (Request* r : s.batch) {
    const size_t b = (size_t)(r->off[r->nt] - r->off[0]);
    if (b) memcpy(hio + pos, r->codes.data() + r->off[0], b);
    pos += b;
  }
  ENSURE(codes, cbytes + 16);
  ENSURE(outK, nel * 4 + 16);
  ENSURE(outKhat, nel * 8 + 16);
  if (want_f) ENSURE(outF, (size_t)nt * 8);
  cudaError_t e = cudaSuccess;
  if (cbytes) e = cudaMemcpyAsync(w.codes.p, hio, cbytes, cudaMemcpyHostToDevice, w.cs);
  if (e != cudaSuccess) return wcuda(w, e, "copy codes to device");
  if ((rc = enqueue_cross(c, w, (const uint8_t*)w.codes.p, off.data(), nt, (int32_t*)w.outK.p,
                          (double*)w.outKhat.p, want_f ? (double*)w.outF.p : nullptr)) != GAKCO_OK)
    return rc;
  e = cudaMemcpyAsync(hio + s.k_off, w.outK.p, nel * 4, cudaMemcpyDeviceToHost, w.cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hio + s.kh_off, w.outKhat.p, nel * 8, cudaMemcpyDeviceToHost, w.cs);
  if (e == cudaSuccess && want_f)
    e = cudaMemcpyAsync(hio + s.f_off, w.outF.p, (size_t)nt * 8, cudaMemcpyDeviceToHost, w.cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_status, w.status.p, 128, cudaMemcpyDeviceToHost, w.cs);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(w.cs, on_slot_done, &s);
  if (e != cudaSuccess) return wcuda(w, e, "enqueue results");
  return GAKCO_OK;
}

// Completion of a slot's batch (no lock held): check, then copy each
// request's rows out of the pinned staging into the caller's buffers.
int complete_batch(gakco_ctx* c, Slot& s) {
  Work& w = s.w;
  cudaError_t e = cudaStreamSynchronize(w.cs);  // returns at once: the callback ran
  if (e != cudaSuccess) return wcuda(w, e, "serving batch");
  int rc = check_status(c, w);
  if (rc != GAKCO_OK) return rc;
  const size_t ntr = (size_t)c->train.n;
  const uint8_t* hio = (const uint8_t*)w.h_io;
  for (size_t i = 0; i < s.batch.size(); ++i) {
    Request* r = s.batch[i];
    const size_t rows = (size_t)r->nt;
    if (r->K) memcpy(r->K, hio + s.k_off + (size_t)s.row0[i] * ntr * 4, rows * ntr * 4);
    if (r->Khat) memcpy(r->Khat, hio + s.kh_off + (size_t)s.row0[i] * ntr * 8, rows * ntr * 8);
    if (r->F) memcpy(r->F, hio + s.f_off + (size_t)s.row0[i] * 8, rows * 8);
  }
  return GAKCO_OK;
}

void finish_requests(gakco_ctx* c, Slot& s, int rc, const std::string& err) {
  const double t = now_ms();
  for (Request* r : s.batch) {
    r->rc = rc;
    r->err = err;
    r->t_done = t;
  }
  c->served_batches += 1;
  c->served_requests += (int64_t)s.batch.size();
  s.batch.clear();
  s.busy = false;
  s.gpu_done.store(false);
}

void dispatcher_main(gakco_ctx* c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  for (;;) {
    bool progressed = false;
    // Completions.
    for (auto& sp : c->slots) {
      Slot& s = *sp;
      if (s.busy && s.gpu_done.load()) {
        lk.unlock();
        const int rc = complete_batch(c, s);
        lk.lock();
        finish_requests(c, s, rc, rc == GAKCO_OK ? std::string() : s.w.err);
        progressed = true;
      }
    }
    if (progressed) c->cv.notify_all();
    // Admissions.
    for (auto& sp : c->slots) {
      Slot& s = *sp;
      if (s.busy || c->pending.empty()) continue;
      size_t busy_bytes = 0;
      bool any_busy = false;
      for (auto& o : c->slots)
        if (o->busy) {
          busy_bytes += o->w.bytes();
          any_busy = true;
        }
      int64_t seqs = 0, wins = 0;
      std::vector<Request*> batch;
      while (!c->pending.empty()) {
        Request* r = c->pending.front();
        if (!batch.empty() &&
            (seqs + r->nt > c->serve_max_seqs || wins + (int64_t)r->windows > c->serve_max_windows))
          break;
        batch.push_back(r);
        seqs += r->nt;
        wins += (int64_t)r->windows;
        c->pending.pop_front();
      }
      // Memory admission: estimated device bytes of this batch.
      const double est = (double)wins * (double)c->masks.size() * 24.0 +
                         (double)seqs * (double)c->train.n * (4.0 * (c->M + 1) + 12.0);
      if (c->serve_mem_bytes > 0 && any_busy && (double)busy_bytes + est > (double)c->serve_mem_bytes) {
        for (auto it = batch.rbegin(); it != batch.rend(); ++it) c->pending.push_front(*it);
        break;  // wait for a slot to free memory
      }
      s.batch = batch;
      s.busy = true;
      s.gpu_done.store(false);
      lk.unlock();
      const int rc = launch_batch(c, s);
      lk.lock();
      if (rc != GAKCO_OK) {
        finish_requests(c, s, rc, s.w.err);
        c->cv.notify_all();
      }
      progressed = true;
    }
    if (c->stopping) {
      bool busy = false;
      for (auto& sp : c->slots) busy |= sp->busy;
      if (!busy) break;
    }
    if (!progressed) c->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

int start_serving(gakco_ctx* c) {
  if (c->serving) return GAKCO_OK;
  for (int i = 0; i < c->serve_slots; ++i) {
    std::unique_ptr<Slot> s(new Slot());
    if (init_work(s->w) != GAKCO_OK) return fail(c, GAKCO_E_CUDA, "serving slot: %s", s->w.err.c_str());
    c->slots.push_back(std::move(s));
  }
  c->stopping = false;
  try {
    c->dispatcher = std::thread(dispatcher_main, c);
  } catch (...) {
    return fail(c, GAKCO_E_INTERNAL, "could not start the serving thread");
  }
  c->serving = true;
  return GAKCO_OK;
}

void stop_serving(gakco_ctx* c) {
  if (!c->serving) return;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->stopping = true;
    for (Request* r : c->pending) {
      r->rc = GAKCO_E_INVALID;
      r->err = "context destroyed before the request ran";
    }
    c->pending.clear();
  }
  c->cv.notify_all();
  c->dispatcher.join();
  for (auto& sp : c->slots) release_work(sp->w);
  c->slots.clear();
  for (auto& kv : c->requests) delete kv.second;
  c->requests.clear();
  c->serving = false;
}

// -------------------------------------------------------------- autotuner --
//
// Picks the sort digit width, the sort chunk size, the accumulation block
// size and the mask-group size for a workload by timing the stages they
// drive (each candidate run once with per-kernel events), one parameter at
// a time; then the dense-level mode (never / cost model / every qualifying
// level) by the time of all stages together.  Choices are cached per (sigma, g, k, SM count, window and
// sequence-count buckets) for the life of the process.

struct TuneChoice {
  int radix_bits;
  int64_t chunk_elems;
  int accum_threads;
  int64_t group_bytes;
  int dense;
  int accum_variant;
  int rle_items;
  int level_bits[kMaxLevels];
};

std::mutex g_tune_mu;
std::unordered_map<uint64_t, TuneChoice> g_tune_cache;

// Time of the named stages of the last profiled call (all stages when
// `a` is null).
double stage_ms(gakco_ctx* c, const char* a, const char* b = nullptr) {
  double t = 0;
  for (auto& kv : c->timings)
    if (!a || kv.first == a || (b && kv.first == b)) t += kv.second.first;
  return t;
}

int autotune(gakco_ctx* c, int32_t nd, const uint8_t* const* codes, const int64_t* const* off,
             const int32_t* n, cudaStream_t user, std::string& report) {
  Work& w = c->main;
  uint64_t G = 0, nmax = 0, nn = 0;
  for (int32_t d = 0; d < nd; ++d) {
    nmax = std::max<uint64_t>(nmax, (uint64_t)n[d]);
    nn += (uint64_t)n[d] * n[d];
    for (int32_t x = 0; x < n[d]; ++x) {
      const int64_t len = off[d][x + 1] - off[d][x];
      if (len >= c->g) G += (uint64_t)(len - c->g + 1);
    }
  }
  auto bucket = [](uint64_t v) {
    int b = 0;
    while (v > 1) {
      v >>= 1;
      ++b;
    }
    return (uint64_t)b;
  };
  const uint64_t key = ((uint64_t)c->sigma << 56) ^ ((uint64_t)c->g << 48) ^ ((uint64_t)c->k << 40) ^
                       ((uint64_t)c->nsm << 28) ^ (bucket(G) << 20) ^ (bucket(nmax) << 12) ^ (uint64_t)nd;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c->radix_bits = it->second.radix_bits;
      c->chunk_elems = it->second.chunk_elems;
      c->accum_threads = it->second.accum_threads;
      c->group_bytes = it->second.group_bytes;
      c->dense = it->second.dense;
      c->accum_variant = it->second.accum_variant;
      c->rle_items = it->second.rle_items;
      memcpy(c->level_bits, it->second.level_bits, sizeof c->level_bits);
      drop_graph(c);
      report = "cached";
      return GAKCO_OK;
    }
  }
  int rc;
  ENSURE(outK, nn * 4 + 16);
  std::vector<int32_t*> Kp(nd);
  uint64_t o = 0;
  for (int32_t d = 0; d < nd; ++d) {
    Kp[d] = (int32_t*)w.outK.p + o;
    o += (uint64_t)n[d] * n[d];
  }
  const int saved_profile = c->profile, saved_engine = c->engine;
  memset(c->level_bits, 0, sizeof c->level_bits);
  c->profile = 1;
  c->engine = 0;
  c->dense = 0;
  auto trial = [&](const char* s1, const char* s2, double& ms) -> int {
    Plan p;
    int r = plan_datasets(c, w, p, nd, codes, off, n, Kp.data(), nullptr, nullptr, true);
    if (r == GAKCO_OK) r = run_gram(c, p, user);
    ms = r == GAKCO_OK ? stage_ms(c, s1, s2) : 1e30;
    return r;
  };
  char buf[256];
  double best, t;
  // Sort digit width (sort + run-length time).
  int best_rb = c->radix_bits;
  best = 1e30;
  for (int rb : {6, 8, 10}) {
    c->radix_bits = rb;
    if ((rc = trial("sort_pass", "run_length", t)) != GAKCO_OK) break;
    if (t < best) best = t, best_rb = rb;
  }
  c->radix_bits = best_rb;
  // Digit width per level: the levels' key widths differ (e.g. 26 bits take
  // four 8-bit passes but three 9-bit ones), so each level may take its
  // own width.
  for (int m = 0; m <= c->M && rc == GAKCO_OK; ++m) {
    if (c->lkbits[m] <= 8) continue;  // one pass at any width
    c->level_bits[m] = 0;
    double best_t;
    if ((rc = trial("sort_pass", "run_length", best_t)) != GAKCO_OK) break;
    int best_b = 0;
    for (int rb : {7, 9, 10, 11}) {
      if (rb == best_rb) continue;
      c->level_bits[m] = rb;
      if ((rc = trial("sort_pass", "run_length", t)) != GAKCO_OK) break;
      if (t < 0.98 * best_t) best_t = t, best_b = rb;  // a clear gain only
    }
    c->level_bits[m] = best_b;
  }
  // Sort chunk size.
  int64_t best_ch = c->chunk_elems;
  best = 1e30;
  for (int64_t ch : {(int64_t)1 << 22, (int64_t)1 << 24, (int64_t)1 << 26}) {
    if (rc != GAKCO_OK) break;
    c->chunk_elems = ch;
    if ((rc = trial("sort_pass", "run_length", t)) != GAKCO_OK) break;
    if (t < best) best = t, best_ch = ch;
  }
  c->chunk_elems = best_ch;
  // Elements per thread of the run-length kernels.
  int best_ri = c->rle_items;
  best = 1e30;
  for (int ri : {16, 8}) {
    if (rc != GAKCO_OK) break;
    c->rle_items = ri;
    if ((rc = trial("run_length", nullptr, t)) != GAKCO_OK) break;
    if (t < best) best = t, best_ri = ri;
  }
  c->rle_items = best_ri;
  // Accumulation block size and mask-group bytes.
  int best_th = c->accum_threads;
  int64_t best_gb = c->group_bytes;
  best = 1e30;
  for (int th : {256, 512}) {
    for (int64_t gb : {(int64_t)64 << 20, (int64_t)128 << 20, (int64_t)256 << 20, (int64_t)512 << 20}) {
      if (rc != GAKCO_OK) break;
      c->accum_threads = th;
      c->group_bytes = gb;
      if ((rc = trial("accumulate", nullptr, t)) != GAKCO_OK) break;
      if (t < best) best = t, best_th = th, best_gb = gb;
    }
  }
  c->accum_threads = best_th;
  c->group_bytes = best_gb;
  // Dense-level mode, by the time of every stage.
  int best_dense = 0;
  best = 1e30;
  for (int dm : {0, 1, 2}) {
    if (rc != GAKCO_OK) break;
    c->dense = dm;
    if ((rc = trial(nullptr, nullptr, t)) != GAKCO_OK) break;
    if (t < best) best = t, best_dense = dm;
  }
  c->dense = best_dense;
  // How the accumulation walks short entry ranges, with the choices above.
  int best_var = c->accum_variant;
  best = 1e30;
  for (int v : {0, 1, 2}) {
    if (rc != GAKCO_OK) break;
    c->accum_variant = v;
    if ((rc = trial("accumulate", nullptr, t)) != GAKCO_OK) break;
    if (t < best) best = t, best_var = v;
  }
  c->accum_variant = best_var;
  c->profile = saved_profile;
  c->engine = saved_engine;
  drop_graph(c);
  if (rc != GAKCO_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneChoice tc{best_rb, best_ch, best_th, best_gb, best_dense, best_var, best_ri, {}};
    memcpy(tc.level_bits, c->level_bits, sizeof tc.level_bits);
    g_tune_cache[key] = tc;
  }
  snprintf(buf, sizeof buf,
           "radix_bits=%d chunk_elems=%lld rle_items=%d accum_threads=%d group_bytes=%lld dense=%d accum_variant=%d",
           best_rb, (long long)best_ch, best_ri, best_th, (long long)best_gb, best_dense, best_var);
  report = buf;
  for (int m = 0; m <= c->M; ++m)
    if (c->level_bits[m]) report += " level" + std::to_string(m) + "_bits=" + std::to_string(c->level_bits[m]);
  return GAKCO_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI --

extern "C" {

int gakco_create(int sigma, int g, int k, gakco_ctx** out) {
  if (!out) return GAKCO_E_INVALID;
  *out = nullptr;
  if (sigma < 2 || sigma > 255 || g < 1 || k < 1 || k > g) return GAKCO_E_INVALID;
  int bits = 0;
  while ((1 << bits) < sigma) ++bits;
  if (g * bits > 64) return GAKCO_E_INVALID;
  const int M = g - k;
  if (M + 1 > kMaxLevels) return GAKCO_E_INVALID;
  uint64_t cgk = 0;
  for (int m = 0; m <= M; ++m) cgk += binom(g, m);
  if (cgk > (1u << 16)) return GAKCO_E_INVALID;

  gakco_ctx* c = new gakco_ctx();
  c->sigma = sigma;
  c->g = g;
  c->k = k;
  c->M = M;
  c->bits = bits;
  // Masks in level order; within a level, deleted position sets in
  // lexicographic order (Alg. 1: for m, for i < C(g, m)).
  // A non-power-of-two alphabet folds the kept symbols in base sigma (see
  // MaskDesc): ceil(log2(sigma^(g-m))) key bits.
  const bool pow2 = (sigma & (sigma - 1)) == 0;
  for (int m = 0; m <= M; ++m) {
    int kw = (g - m) * bits;
    if (!pow2) {
      uint64_t v = 1;
      for (int i = 0; i < g - m; ++i) v *= (uint64_t)sigma;  // < 2^(bits (g-m)) <= 2^64
      kw = v > 1 ? 64 - __builtin_clzll(v - 1) : 1;
    }
    c->lkbits[m] = kw;
  }
  for (int m = 0; m <= M; ++m) {
    std::vector<int> del(m);
    for (int i = 0; i < m; ++i) del[i] = i;
    for (;;) {
      std::vector<int> keep;
      for (int q = 0, j = 0; q < g; ++q) {
        if (j < m && del[j] == q)
          ++j;
        else
          keep.push_back(q);
      }
      MaskDesc md{};
      md.level = (uint32_t)m;
      md.kbits = (uint32_t)c->lkbits[m];
      const int nk = (int)keep.size();
      if (!pow2) {
        md.fold = (uint32_t)sigma;
        md.nkeep = (uint32_t)nk;
        md.symmask = (1u << bits) - 1;
        for (int j = 0; j < nk; ++j) md.ksh[j] = (uint8_t)(bits * (g - 1 - keep[j]));
      }
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
      c->masks.push_back(md);
      c->mask_level.push_back((uint32_t)m);
      int i = m - 1;
      while (i >= 0 && del[i] == g - m + i) --i;
      if (i < 0) break;
      del[i]++;
      for (int j = i + 1; j < m; ++j) del[j] = del[j - 1] + 1;
    }
  }
  for (int m = 0; m <= M; ++m) {
    c->h[m] = (uint32_t)binom(g - m, k);                                       // Eq. 6
    for (int j = 0; j < m; ++j) c->ie[m][j] = (uint32_t)binom(g - j, m - j);  // Eq. 9
    c->maxC = std::max<uint32_t>(c->maxC, (uint32_t)binom(g, m));
  }

  cudaError_t e = cudaGetDevice(&c->device);
  int v = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->smem_optin = (size_t)v;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = (cudaError_t)prep_init();
  if (e == cudaSuccess) e = (cudaError_t)dense_init();
  if (e == cudaSuccess) {
    size_t fr = 0, tot = 0;
    int ats = 0, pma = 0;
    if (cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, c->device) == cudaSuccess &&
        cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, c->device) == cudaSuccess)
      c->pageable_ats = pma == 1 && ats == 1;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && tot > 0)
    {
      c->dense_bytes = std::min<int64_t>(c->dense_bytes, (int64_t)(tot / 4));
      c->heavy_bytes = std::min<int64_t>(c->heavy_bytes, (int64_t)(tot / 16));
    }
    cudaGetLastError();
  }
  if (e == cudaSuccess && init_work(c->main) != GAKCO_OK) e = cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    cudaGetLastError();
    gakco_destroy(c);
    return GAKCO_E_CUDA;
  }
  *out = c;
  return GAKCO_OK;
}

void gakco_destroy(gakco_ctx* c) {
  if (!c) return;
  stop_serving(c);
  if (c->main.cs) cudaStreamSynchronize(c->main.cs);
  drop_graph(c);
  release_work(c->main);
  for (Train* T : {&c->train, &c->train_add, &c->train_merged}) {
    DevBuf* tb[] = {&T->ukey, &T->ufirst, &T->eseq, &T->nfeat, &T->diagC, &T->rinv, &T->svm, &T->tcodes};
    for (DevBuf* b : tb) release(*b);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  delete c;
}

const char* gakco_last_error(const gakco_ctx* c) { return c ? c->err.c_str() : "null context"; }

int gakco_set_option(gakco_ctx* c, int key, int64_t v) {
  if (!c) return GAKCO_E_INVALID;
  switch (key) {
    case GAKCO_OPT_ENGINE:
      if (v != 0 && v != 1) return fail(c, GAKCO_E_INVALID, "engine must be 0 or 1");
      c->engine = (int)v;
      break;
    case GAKCO_OPT_RADIX_BITS:
      if (v < 4 || v > kMaxRadixBits) return fail(c, GAKCO_E_INVALID, "radix bits must be 4..%d", kMaxRadixBits);
      c->radix_bits = (int)v;
      break;
    case GAKCO_OPT_CHUNK_ELEMS:
      if (v < kTile) return fail(c, GAKCO_E_INVALID, "chunk must hold >= %d elements", kTile);
      c->chunk_elems = v;
      break;
    case GAKCO_OPT_GRAPH:
      c->use_graph = v != 0;
      break;
    case GAKCO_OPT_ACCUM_THREADS:
      if (v != 256 && v != 512 && v != 1024) return fail(c, GAKCO_E_INVALID, "threads must be 256, 512 or 1024");
      c->accum_threads = (int)v;
      break;
    case GAKCO_OPT_PROFILE:
      c->profile = v != 0;
      break;
    case GAKCO_OPT_SMEM_COLS:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "column cap must be >= 0");
      c->smem_cols = v;
      break;
    case GAKCO_OPT_FAIL_ALLOC_AFTER:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "allocation countdown must be >= 0");
      c->fail_alloc_after = v;
      break;
    case GAKCO_OPT_GROUP_BYTES:
      if (v < 1) return fail(c, GAKCO_E_INVALID, "group bytes must be >= 1");
      c->group_bytes = v;
      break;
    case GAKCO_OPT_SERVE_SLOTS:
      if (v < 1 || v > 16) return fail(c, GAKCO_E_INVALID, "serving slots must be 1..16");
      if (c->serving) return fail(c, GAKCO_E_INVALID, "serving already started");
      c->serve_slots = (int)v;
      break;
    case GAKCO_OPT_SERVE_MAX_SEQS:
      if (v < 1 || v > 65535) return fail(c, GAKCO_E_INVALID, "batch sequences must be 1..65535");
      c->serve_max_seqs = v;
      break;
    case GAKCO_OPT_SERVE_MAX_WINDOWS:
      if (v < 1) return fail(c, GAKCO_E_INVALID, "batch windows must be >= 1");
      c->serve_max_windows = v;
      break;
    case GAKCO_OPT_SERVE_MEM_BYTES:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "memory budget must be >= 0");
      c->serve_mem_bytes = v;
      break;
    case GAKCO_OPT_DENSE:
      if (v < 0 || v > 2) return fail(c, GAKCO_E_INVALID, "dense mode must be 0, 1 or 2");
      c->dense = (int)v;
      break;
    case GAKCO_OPT_DENSE_BYTES:
      if (v < 1) return fail(c, GAKCO_E_INVALID, "dense bytes must be >= 1");
      c->dense_bytes = v;
      break;
    case GAKCO_OPT_OVERLAP:
      if (v != 0 && v != 1) return fail(c, GAKCO_E_INVALID, "overlap must be 0 or 1");
      c->overlap = (int)v;
      break;
    case GAKCO_OPT_HEAVY:
      if (v < 0 || v > 1000) return fail(c, GAKCO_E_INVALID, "heavy threshold must be 0..1000 (thousandths)");
      c->heavy = (int)v;
      break;
    case GAKCO_OPT_DIRECT_D2H:
      if (v < -1 || v > 1) return fail(c, GAKCO_E_INVALID, "direct copies must be -1, 0 or 1");
      c->direct_d2h = (int)v;
      break;
    case GAKCO_OPT_HEAVY_BYTES:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "heavy bytes must be >= 0");
      c->heavy_bytes = v;
      break;
    case GAKCO_OPT_DENSE_SMS:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "dense SM count must be >= 0");
      c->dense_sms = (int)v;
      break;
    case GAKCO_OPT_KERNEL_ONLY:
      if (v != 0 && v != 1) return fail(c, GAKCO_E_INVALID, "kernel-only must be 0 or 1");
      c->kernel_only = (int)v;
      break;
    case GAKCO_OPT_DENSE_RUN_COLS:
      if (v < 128) return fail(c, GAKCO_E_INVALID, "dense run columns must be >= 128");
      c->dense_run_cols = v;
      break;
    case GAKCO_OPT_ACCUM_VARIANT:
      if (v < 0 || v > 2) return fail(c, GAKCO_E_INVALID, "accumulation variant must be 0, 1 or 2");
      c->accum_variant = (int)v;
      break;
    case GAKCO_OPT_LEVEL_RADIX_BITS: {
      const int64_t m = v >> 8, b = v & 0xFF;
      if (m < 0 || m > c->M || (b != 0 && (b < 4 || b > kMaxRadixBits)))
        return fail(c, GAKCO_E_INVALID, "level digit width: (level << 8) | bits, level 0..M, bits 0 or 4..%d",
                    kMaxRadixBits);
      c->level_bits[m] = (int)b;
      break;
    }
    case GAKCO_OPT_DENSE_LATE:
      if (v != 0 && v != 1) return fail(c, GAKCO_E_INVALID, "dense late must be 0 or 1");
      c->dense_late = (int)v;
      break;
    case GAKCO_OPT_DENSE_SPLIT:
      if (v < -1 || v > 1) return fail(c, GAKCO_E_INVALID, "dense split must be -1, 0 or 1");
      c->dense_split = (int)v;
      break;
    case GAKCO_OPT_RLE_ITEMS:
      if (v != 8 && v != 16) return fail(c, GAKCO_E_INVALID, "run-length items must be 8 or 16");
      c->rle_items = (int)v;
      break;
    case GAKCO_OPT_SORT:
      if (v != 0 && v != 1) return fail(c, GAKCO_E_INVALID, "sort must be 0 or 1");
      c->sort_mode = (int)v;
      break;
    case GAKCO_OPT_DENSE_ROUND_SUM:
      if (v < 1 || v > (int64_t)kDenseExactSum)
        return fail(c, GAKCO_E_INVALID, "dense round sum must be 1..%u", kDenseExactSum);
      c->dense_round_sum = v;
      break;
    case GAKCO_OPT_DENSE_WAIT_CYCLES:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "dense wait cycles must be >= 0");
      c->dense_wait_cycles = v;
      break;
    case GAKCO_OPT_DENSE_OVERFLOW:
      if (v < 1 || v > ((int64_t)1 << 26)) return fail(c, GAKCO_E_INVALID, "overflow entries must be 1..2^26");
      c->dense_overflow = v;
      break;
    default:
      return fail(c, GAKCO_E_INVALID, "unknown option %d", key);
  }
  drop_graph(c);
  return GAKCO_OK;
}

int gakco_get_stat(const gakco_ctx* c, int key, double* v) {
  if (!c || !v) return GAKCO_E_INVALID;
  gakco_ctx* cc = const_cast<gakco_ctx*>(c);
  switch (key) {
    case GAKCO_STAT_LAUNCHES:
      *v = (double)c->last_launches;
      return GAKCO_OK;
    case GAKCO_STAT_MASK_PASSES:
      *v = (double)c->last_mask_passes;
      return GAKCO_OK;
    case GAKCO_STAT_DEVICE_BYTES: {
      double s = (double)cc->main.bytes();
      for (const Train* T : {&c->train, &c->train_add, &c->train_merged})
        s += (double)(T->ukey.cap + T->ufirst.cap + T->eseq.cap + T->nfeat.cap + T->diagC.cap + T->rinv.cap +
                      T->tcodes.cap);
      std::lock_guard<std::mutex> lk(cc->mu);
      for (auto& sp : cc->slots) s += (double)sp->w.bytes();
      *v = s;
      return GAKCO_OK;
    }
    case GAKCO_STAT_GRAPH_REPLAY:
      *v = c->last_replay;
      return GAKCO_OK;
    case GAKCO_STAT_PAIR_UPDATES:
      *v = c->last_pairs;
      return GAKCO_OK;
    case GAKCO_STAT_ENTRIES_VISITED:
      *v = c->last_entries;
      return GAKCO_OK;
    case GAKCO_STAT_WINDOWS_VISITED:
      *v = c->last_windows;
      return GAKCO_OK;
    case GAKCO_STAT_DENSE_PROBLEMS:
      *v = c->plan_dense_probs;
      return GAKCO_OK;
    case GAKCO_STAT_DENSE_FLOPS:
      *v = c->plan_dense_flops;
      return GAKCO_OK;
    case GAKCO_STAT_DENSE_ISSUED_FLOPS:
      *v = c->plan_dense_issued;
      return GAKCO_OK;
    case GAKCO_STAT_DENSE_BYTES:
      *v = c->plan_dense_bytes;
      return GAKCO_OK;
    case GAKCO_STAT_HEAVY_COLUMNS:
      *v = c->last_heavy_cols;
      return GAKCO_OK;
    case GAKCO_STAT_HEAVY_FLOPS:
      *v = c->last_heavy_flops;
      return GAKCO_OK;
    case GAKCO_STAT_MASKS:
      *v = (double)c->masks.size();
      return GAKCO_OK;
    case GAKCO_STAT_RLE_BYTES:
      *v = c->plan_rle_bytes + 8.0 * c->last_rle_entries;
      return GAKCO_OK;
    case GAKCO_STAT_PACK_BYTES:
      *v = c->plan_pack_bytes;
      return GAKCO_OK;
    case GAKCO_STAT_COMBINE_BYTES:
      *v = c->plan_combine_bytes;
      return GAKCO_OK;
    case GAKCO_STAT_SORT_BYTES:
      *v = c->plan_sort_bytes;
      return GAKCO_OK;
    case GAKCO_STAT_SERVED_BATCHES: {
      std::lock_guard<std::mutex> lk(cc->mu);
      *v = (double)c->served_batches;
      return GAKCO_OK;
    }
    case GAKCO_STAT_SERVED_REQUESTS: {
      std::lock_guard<std::mutex> lk(cc->mu);
      *v = (double)c->served_requests;
      return GAKCO_OK;
    }
  }
  return GAKCO_E_INVALID;
}

int gakco_kernel_timing(const gakco_ctx* c, int idx, char* name, int name_len, double* ms,
                        int64_t* launches) {
  if (!c || idx < 0 || (size_t)idx >= c->timings.size()) return GAKCO_E_INVALID;
  const auto& kv = c->timings[idx];
  if (name && name_len > 0) snprintf(name, (size_t)name_len, "%s", kv.first.c_str());
  if (ms) *ms = kv.second.first;
  if (launches) *launches = kv.second.second;
  return GAKCO_OK;
}

int gakco_gram(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t n, int32_t* K,
               double* Khat, int32_t* Nm) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  return ret(c, c->main, gram_host(c, 1, &codes, &offsets, &n, &K, &Khat, &Nm));
}

int gakco_gram_batch(gakco_ctx* c, int32_t nd, const uint8_t* const* codes,
                     const int64_t* const* offsets, const int32_t* n, int32_t* const* K,
                     double* const* Khat, int32_t* const* Nm) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  return ret(c, c->main, gram_host(c, nd, codes, offsets, n, K, Khat, Nm));
}

int gakco_gram_batch_device(gakco_ctx* c, int32_t nd, const uint8_t* const* codes,
                            const int64_t* const* offsets, const int32_t* n, int32_t* const* K,
                            double* const* Khat, int32_t* const* Nm, void* stream) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  Plan p;
  int rc = plan_datasets(c, c->main, p, nd, codes, offsets, n, K, Khat, Nm, true);
  if (rc == GAKCO_OK) rc = run_gram(c, p, (cudaStream_t)stream);
  return ret(c, c->main, rc);
}

int gakco_gram_device(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t n,
                      int32_t* K, double* Khat, int32_t* Nm, void* stream) {
  return gakco_gram_batch_device(c, 1, &codes, &offsets, &n, &K, &Khat, &Nm, stream);
}

int gakco_gram_partial_device(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t n,
                              int32_t mask_begin, int32_t mask_end, uint32_t* C, void* stream) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  const int32_t nmask = (int32_t)c->masks.size();
  if (mask_begin < 0 || mask_end < mask_begin || mask_end > nmask)
    return fail(c, GAKCO_E_INVALID, "mask slice [%d, %d) outside [0, %d)", mask_begin, mask_end, nmask);
  if (c->engine != 0) return fail(c, GAKCO_E_INVALID, "partial Gram calls need the batched engine");
  if (n > 0 && !C) return fail(c, GAKCO_E_INVALID, "partial Gram calls need a C buffer");
  Plan p;
  int32_t* kk = (int32_t*)C;  // passes the device-call check; no K is written
  int rc = plan_datasets(c, c->main, p, 1, &codes, &offsets, &n, &kk, nullptr, nullptr, true);
  if (rc == GAKCO_OK) {
    for (DsHost& D : p.ds) D.K = nullptr;
    p.mask_lo = (uint32_t)mask_begin;
    p.mask_hi = (uint32_t)mask_end;
    p.partial_C = C;
    if (n > 0 && mask_end == mask_begin) {
      // An empty slice adds nothing: its C is all zero.
      cudaError_t e = cudaMemsetAsync(C, 0, (size_t)(c->M + 1) * n * n * 4, (cudaStream_t)stream);
      if (e != cudaSuccess) return ret(c, c->main, wcuda(c->main, e, "clear C"));
      c->last_mask_passes = 0;
      c->last_launches = 0;
      return GAKCO_OK;
    }
    rc = run_gram(c, p, (cudaStream_t)stream);
  }
  return ret(c, c->main, rc);
}

int gakco_combine_device(gakco_ctx* c, const uint32_t* C, int32_t n, int32_t* K, double* Khat,
                         int32_t* Nm, void* stream) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  if (n < 0 || n > 65535) return fail(c, GAKCO_E_INVALID, "n = %d outside [0, 65535]", n);
  if (n == 0) return GAKCO_OK;
  if (!C || !K) return fail(c, GAKCO_E_INVALID, "combine needs C and K");
  Work& w = c->main;
  int rc;
  // The table area and the norms buffer are rewritten: a cached Gram graph
  // would replay with them.
  drop_graph(c);
  auto run = [&]() -> int {
    ENSURE(rinv, (size_t)n * 8);
    ENSURE(status, 128);
    Tables t;
    DsInfo in{};
    in.K = K;
    in.Nm = Nm;
    in.Khat = Khat;
    in.rinv = (double*)w.rinv.p;
    in.C = const_cast<uint32_t*>(C);
    in.n = (uint32_t)n;
    const size_t o_info = t.add(&in, sizeof in);
    if ((rc = upload_tables(c, w, t)) != GAKCO_OK) return rc;
    cudaStream_t user = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(c->ev_in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w.cs, c->ev_in, 0);
    if (e != cudaSuccess) return wcuda(w, e, "stream ordering");
    cudaMemsetAsync(w.status.p, 0, 128, w.cs);
    c->timed.clear();
    c->ev_used = 0;
    AccParams a{};  // the tail kernels read only the coefficients and the status word
    a.M = (uint32_t)c->M;
    a.status = (uint32_t*)w.status.p;
    memcpy(a.h, c->h, sizeof a.h);
    memcpy(a.ie, c->ie, sizeof a.ie);
    const DsInfo* d_info = (const DsInfo*)((uint8_t*)w.tables.p + o_info);
    const uint32_t nt = (uint32_t)((n + 31) / 32);
    launch_diag(d_info, 1, (uint32_t)n, a, w.cs);
    launch_combine(d_info, 1, nt * nt, a, Nm != nullptr, Khat != nullptr, w.cs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return wcuda(w, e, "kernel launch");
    c->last_launches = 2;
    rc = sync_and_check(c, w);
    e = cudaEventRecord(c->ev_out, w.cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, c->ev_out, 0);
    if (e != cudaSuccess && rc == GAKCO_OK) rc = wcuda(w, e, "stream ordering");
    return rc;
  };
  return ret(c, w, run());
}

int gakco_autotune(gakco_ctx* c, int32_t nd, const uint8_t* const* codes,
                   const int64_t* const* offsets, const int32_t* n, void* stream, char* report,
                   int report_len) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  if (nd < 1 || !codes || !offsets || !n) return fail(c, GAKCO_E_INVALID, "autotune needs datasets");
  std::string rep;
  const int rc = autotune(c, nd, codes, offsets, n, (cudaStream_t)stream, rep);
  if (report && report_len > 0) snprintf(report, (size_t)report_len, "%s", rep.c_str());
  return ret(c, c->main, rc);
}

int gakco_fit(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t n) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    bool busy = !c->pending.empty();
    for (auto& sp : c->slots) busy |= sp->busy;
    if (busy) return fail(c, GAKCO_E_INVALID, "requests are in flight; wait for them before fitting");
  }
  Work& w = c->main;
  if (n < 0 || n > 65535 || (n > 0 && !offsets)) return fail(c, GAKCO_E_INVALID, "bad training set");
  const uint64_t cbytes = n > 0 ? (uint64_t)offsets[n] : 0;
  int rc = ensure(c, w, w.codes, cbytes + 16, "codes");
  if (rc != GAKCO_OK) return ret(c, w, rc);
  if (cbytes) {
    cudaError_t e = cudaMemcpyAsync(w.codes.p, codes, cbytes, cudaMemcpyHostToDevice, w.cs);
    if (e != cudaSuccess) return ret(c, w, wcuda(w, e, "copy codes to device"));
  }
  return ret(c, w, fit(c, (const uint8_t*)w.codes.p, offsets, n));
}

int gakco_fit_device(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t n,
                     void* stream) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    bool busy = !c->pending.empty();
    for (auto& sp : c->slots) busy |= sp->busy;
    if (busy) return fail(c, GAKCO_E_INVALID, "requests are in flight; wait for them before fitting");
  }
  Work& w = c->main;
  cudaError_t e = cudaEventRecord(c->ev_in, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w.cs, c->ev_in, 0);
  if (e != cudaSuccess) return ret(c, w, wcuda(w, e, "stream ordering"));
  return ret(c, w, fit(c, codes, offsets, n));
}

int gakco_cross_fitted(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t nt,
                       int32_t* K, double* Khat) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  return ret(c, c->main, cross_host(c, codes, offsets, nt, K, Khat));
}

int gakco_set_svm(gakco_ctx* c, const double* coef, int32_t n, double bias, int kind) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    bool busy = !c->pending.empty();
    for (auto& sp : c->slots) busy |= sp->busy;
    if (busy) return fail(c, GAKCO_E_INVALID, "requests are in flight; wait for them before setting coefficients");
  }
  Train& T = c->train;
  if (!T.ok) return fail(c, GAKCO_E_INVALID, "no training set: call gakco_fit first");
  if (n != T.n) return fail(c, GAKCO_E_INVALID, "%d coefficients for %d training sequences", n, T.n);
  if (kind != 0 && kind != 1) return fail(c, GAKCO_E_INVALID, "kernel kind must be 0 (Khat) or 1 (K)");
  if (n > 0 && !coef) return fail(c, GAKCO_E_INVALID, "null coefficients");
  Work& w = c->main;
  int rc = ensure(c, w, T.svm, (size_t)std::max(n, 1) * 8, "svm coefficients");
  if (rc != GAKCO_OK) return ret(c, w, rc);
  cudaError_t e = cudaSuccess;
  if (n > 0) e = cudaMemcpyAsync(T.svm.p, coef, (size_t)n * 8, cudaMemcpyHostToDevice, w.cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w.cs);
  if (e != cudaSuccess) return ret(c, w, wcuda(w, e, "copy coefficients"));
  T.svm_bias = bias;
  T.svm_kind = kind;
  T.svm_ok = true;
  return GAKCO_OK;
}

int gakco_extend(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t nb,
                 int32_t* K_rows, double* Khat_rows) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    bool busy = !c->pending.empty();
    for (auto& sp : c->slots) busy |= sp->busy;
    if (busy) return fail(c, GAKCO_E_INVALID, "requests are in flight; wait for them before extending");
  }
  return ret(c, c->main, extend(c, codes, offsets, nb, K_rows, Khat_rows));
}

int gakco_decision(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t nt,
                   double* decision) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  if (nt > 0 && !decision) return fail(c, GAKCO_E_INVALID, "null decision buffer");
  return ret(c, c->main, cross_host(c, codes, offsets, nt, nullptr, nullptr, decision));
}

int gakco_cross_fitted_device(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets,
                              int32_t nt, int32_t* K, double* Khat, void* stream) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  Work& w = c->main;
  if (nt < 0 || nt > 65535 || (nt > 0 && (!offsets || !K))) return fail(c, GAKCO_E_INVALID, "bad test batch");
  if (nt == 0) return GAKCO_OK;
  cudaError_t e = cudaEventRecord(c->ev_in, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w.cs, c->ev_in, 0);
  if (e != cudaSuccess) return ret(c, w, wcuda(w, e, "stream ordering"));
  int rc = enqueue_cross(c, w, codes, offsets, nt, K, Khat);
  if (rc == GAKCO_OK) rc = sync_and_check(c, w);
  if (rc == GAKCO_OK) {
    e = cudaEventRecord(c->ev_out, w.cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, c->ev_out, 0);
    if (e != cudaSuccess) rc = wcuda(w, e, "stream ordering");
  }
  return ret(c, w, rc);
}

int gakco_cross(gakco_ctx* c, const uint8_t* test_codes, const int64_t* test_off, int32_t nt,
                const uint8_t* train_codes, const int64_t* train_off, int32_t ntr, int32_t* K,
                double* Khat) {
  int rc = gakco_fit(c, train_codes, train_off, ntr);
  if (rc != GAKCO_OK) return rc;
  return gakco_cross_fitted(c, test_codes, test_off, nt, K, Khat);
}

int gakco_submit(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t nt,
                 int32_t* K, double* Khat, uint64_t* ticket) {
  return gakco_submit_svm(c, codes, offsets, nt, K, Khat, nullptr, ticket);
}

int gakco_submit_svm(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t nt,
                     int32_t* K, double* Khat, double* decision, uint64_t* ticket) {
  if (!c || !ticket) return GAKCO_E_INVALID;
  if (nt < 1 || nt > 65535 || !offsets) return GAKCO_E_INVALID;
  if (!c->train.ok) return GAKCO_E_INVALID;
  if (decision) {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->train.svm_ok) return fail(c, GAKCO_E_INVALID, "no SVM coefficients: call gakco_set_svm first");
  }
  std::unique_ptr<Request> r(new Request());
  r->nt = nt;
  r->off.assign(offsets, offsets + nt + 1);
  for (int32_t x = 0; x < nt; ++x)
    if (r->off[x] < 0 || r->off[x + 1] < r->off[x]) return GAKCO_E_INVALID;
  if (r->off[nt] > 0 && !codes) return GAKCO_E_INVALID;
  if (r->off[nt] > 0) r->codes.assign(codes, codes + r->off[nt]);
  r->windows = req_windows(c, r.get());
  r->K = K;
  r->Khat = Khat;
  r->F = decision;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->serving) {
    const int rc = start_serving(c);
    if (rc != GAKCO_OK) return rc;
  }
  r->ticket = c->next_ticket++;
  *ticket = r->ticket;
  c->requests[r->ticket] = r.get();
  c->pending.push_back(r.release());
  c->cv.notify_all();
  return GAKCO_OK;
}

int gakco_poll(gakco_ctx* c, uint64_t ticket, int timeout_ms, double* latency_ms) {
  if (!c) return GAKCO_E_INVALID;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->requests.find(ticket);
  if (it == c->requests.end()) return GAKCO_E_INVALID;
  Request* r = it->second;
  if (r->rc > 0 && timeout_ms != 0) {
    auto done = [&] { return r->rc <= 0; };
    if (timeout_ms < 0)
      c->cv.wait(lk, done);
    else
      c->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  }
  if (r->rc > 0) return GAKCO_E_PENDING;
  const int rc = r->rc;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  if (rc != GAKCO_OK) c->err = r->err;
  c->requests.erase(it);
  delete r;
  return rc;
}

}  // extern "C"
