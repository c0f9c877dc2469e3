// Host side of the engine: the C ABI of include/gakco.h, input validation,
// the work plan, device memory, CUDA-graph replay and timing.
//
// The work of one call (Alg. 1 of GaKCo, arXiv 1704.07468):
//   1. pack every window of every dataset into a full g-mer key;
//   2. for every level m and mask, sort the masked keys and count runs
//      (batched: all (dataset, mask) segments of a chunk per launch);
//   3. accumulate C_0..C_M row by row on chip and apply Eq. 9 and Eq. 7;
//   4. mirror the symmetric result and normalise.
// The plain engine instead runs one (dataset, mask) segment per launch and
// applies countAndUpdate with global atomics, as the paper states it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
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

}  // namespace

struct gakco_ctx {
  int sigma = 0, g = 0, k = 0, M = 0, bits = 0;
  std::vector<MaskDesc> masks;
  std::vector<uint32_t> mask_level;
  uint32_t h[kMaxLevels] = {};
  uint32_t ie[kMaxLevels][kMaxLevels] = {};
  uint32_t maxC = 0;  // max_m C(g, m), m <= M

  // options
  int engine = 0;
  int radix_bits = 8;
  int64_t chunk_elems = (int64_t)1 << 24;
  int use_graph = 1;
  int accum_threads = 512;
  int profile = 0;
  int64_t smem_cols = 0;
  int64_t fail_alloc_after = 0;
  int64_t group_bytes = (int64_t)64 << 20;

  std::string err;
  int device = 0;
  int nsm = 0;
  size_t smem_optin = 0;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  DevBuf fullkey, win2seq, ewin, eseq, efe, keyA, keyB, valA, valB, hist, tcnt,
      segtot, estart, etseq, efid, fstart, tables, codes, outK, outKhat, outNm,
      rinv, status, Cplain, Cacc;
  void* h_tables = nullptr;
  size_t h_tables_cap = 0;
  void* h_status = nullptr;

  cudaGraphExec_t gexec = nullptr;
  uint64_t gkey = 0;

  int64_t launches = 0;
  int64_t last_launches = 0, last_mask_passes = 0;
  int last_replay = 0;
  double last_pairs = 0, last_entries = 0, last_windows = 0;
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> timings;
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

int cuda_fail(gakco_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(c, GAKCO_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ensure(gakco_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (bytes <= b.cap) return GAKCO_OK;
  if (c->fail_alloc_after > 0 && --c->fail_alloc_after == 0)
    return fail(c, GAKCO_E_OOM, "injected allocation failure (%s, %zu bytes)", what, bytes);
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
    return fail(c, GAKCO_E_OOM, "cudaMalloc(%s, %zu bytes): %s", what, want, cudaGetErrorString(e));
  }
  b.cap = want;
  return GAKCO_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

void drop_graph(gakco_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey = 0;
}

// Kernel-launch bracket: counts launches and, when profiling, records
// events around them on the engine's stream.
struct Bracket {
  gakco_ctx* c;
  const char* name;
  size_t ia = 0;
  Bracket(gakco_ctx* c_, const char* n_, int count) : c(c_), name(n_) {
    c->launches += count;
    if (c->profile) {
      while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
      }
      ia = c->ev_used;
      c->ev_used += 2;
      cudaEventRecord(c->ev_pool[ia], c->cs);
    }
  }
  ~Bracket() {
    if (c->profile) {
      cudaEventRecord(c->ev_pool[ia + 1], c->cs);
      c->timed.push_back({name, c->ev_pool[ia], c->ev_pool[ia + 1]});
    }
  }
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
  bool any_wide = false;
  uint32_t ncols = 0;
  size_t acc_smem = 0;
  int acc_blocks = 0;
  uint64_t c_elems = 0;
  std::vector<uint32_t> seg_ds;  // dataset of each segment
  bool want_nm = false, want_khat = false;
  // device table offsets
  size_t o_masks, o_level, o_pack, o_info, o_segs, o_tiles, o_items;
  std::vector<size_t> o_coff, o_woff;
};

// Validate datasets and compute window offsets; fills p.ds.
int plan_datasets(gakco_ctx* c, Plan& p, int32_t nd, const uint8_t* const* codes,
                  const int64_t* const* off, const int32_t* n, int32_t* const* K,
                  double* const* Khat, int32_t* const* Nm, bool device) {
  if (nd < 0) return fail(c, GAKCO_E_INVALID, "ndata must be >= 0");
  if (nd > 0 && (!codes || !off || !n)) return fail(c, GAKCO_E_INVALID, "null dataset arrays");
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
      return fail(c, GAKCO_E_INVALID, "dataset %d: n = %d outside [0, 65535]", d, D.n);
    if (D.n > 0 && !D.off) return fail(c, GAKCO_E_INVALID, "dataset %d: null offsets", d);
    if (device && D.n > 0 && !D.K)
      return fail(c, GAKCO_E_INVALID, "dataset %d: device calls need a K buffer", d);
    D.woff.assign(D.n + 1, 0);
    uint64_t acc = 0;
    int64_t total = 0;
    for (int32_t x = 0; x < D.n; ++x) {
      const int64_t len = D.off[x + 1] - D.off[x];
      if (D.off[x] < 0 || len < 0)
        return fail(c, GAKCO_E_INVALID, "dataset %d: offsets must be non-negative and non-decreasing", d);
      const uint64_t W = len >= c->g ? (uint64_t)(len - c->g + 1) : 0;
      wmax = std::max(wmax, W);
      acc += W;
      total += len;
      if (acc >= 0xFFFFFFFFull)
        return fail(c, GAKCO_E_OVERFLOW, "dataset %d: 2^32 or more windows", d);
      D.woff[x + 1] = (uint32_t)acc;
    }
    if (D.n > 0 && total > 0 && !D.codes) return fail(c, GAKCO_E_INVALID, "dataset %d: null codes", d);
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
  const long double bound = (long double)c->maxC * (long double)wmax * (long double)wmax;
  if (bound >= 2147483648.0L)
    return fail(c, GAKCO_E_OVERFLOW,
                "C(g,m) * W_max^2 = %.0Lf reaches 2^31 (W_max = %llu windows); int32 kernel would overflow",
                bound, (unsigned long long)wmax);
  return GAKCO_OK;
}

// Chunks of (dataset, mask) segments, all of one level per chunk.
void plan_chunks(gakco_ctx* c, Plan& p, bool plain) {
  const uint64_t limit = plain ? 0 : (uint64_t)std::max<int64_t>(c->chunk_elems, kTile);
  for (int m = 0; m <= c->M; ++m) {
    const int kb = (c->g - m) * c->bits;
    const int np = (kb + c->radix_bits - 1) / c->radix_bits;
    const int rb = (kb + np - 1) / np;
    std::vector<std::pair<int, int>> passes;
    for (int q = 0; q < np; ++q) passes.push_back({q * rb, std::min(rb, kb - q * rb)});
    const bool wide = kb > 32;
    p.any_wide |= wide;
    Chunk cur{};
    auto flush = [&]() {
      if (cur.nseg == 0) return;
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
      if ((int)c->mask_level[mu] != m) continue;
      for (size_t d = 0; d < p.ds.size(); ++d) {
        const DsHost& D = p.ds[d];
        if (D.G == 0) continue;
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

// Work items of the accumulation kernel: (dataset, level, first mask, mask
// count, row, c0, c1).  The masks of a level are cut into groups whose
// entry arrays (about 12 bytes per window per mask) fit `group_bytes`, so
// the rows processed together share an L2-resident working set; items go
// out group by group, most expensive rows first within a group.
void plan_items(gakco_ctx* c, Plan& p) {
  size_t avail = c->smem_optin > 2048 ? c->smem_optin - 1024 : 0;
  uint32_t ncols = (uint32_t)std::min<size_t>(avail / 4 - 1, 65535);
  if (c->smem_cols > 0) ncols = std::min<uint32_t>(ncols, (uint32_t)c->smem_cols);
  ncols = std::max<uint32_t>(1, std::min<uint32_t>(ncols, std::max<uint32_t>(p.nmax, 1)));
  p.ncols = ncols;
  p.acc_smem = 4 * ((size_t)ncols + 1);  // + the trash slot
  std::vector<uint32_t> level_first(c->M + 2, 0);
  for (uint32_t mu = 0; mu < c->masks.size(); ++mu) level_first[c->mask_level[mu] + 1] = mu + 1;
  for (int m = 1; m <= c->M + 1; ++m) level_first[m] = std::max(level_first[m], level_first[m - 1]);
  struct Row {
    double cost;
    uint32_t x, c0, c1;
  };
  p.items.clear();
  for (size_t d = 0; d < p.ds.size(); ++d) {
    const DsHost& D = p.ds[d];
    if (D.n == 0) continue;
    std::vector<Row> rows;
    for (int32_t x = 0; x < D.n; ++x) {
      const double W = (double)(D.woff[x + 1] - D.woff[x]);
      for (uint32_t t0 = 0; t0 < (uint32_t)D.n; t0 += ncols) {
        const uint32_t t1 = std::min<uint32_t>((uint32_t)D.n, t0 + ncols);
        if (t1 <= (uint32_t)x) continue;
        const uint32_t c0 = std::max<uint32_t>((uint32_t)x, t0);
        rows.push_back({W * (double)(t1 - c0) + W + (double)(t1 - c0), (uint32_t)x, c0, t1});
      }
    }
    std::stable_sort(rows.begin(), rows.end(),
                     [](const Row& a, const Row& b) { return a.cost > b.cost; });
    // Rows without windows still need their (zero) row of C: they are
    // covered by the memset; only rows with windows get items.
    const double per_mask = 12.0 * (double)std::max<uint64_t>(D.G, 1);
    const uint32_t gmax = (uint32_t)std::max(1.0, std::floor((double)c->group_bytes / per_mask));
    for (int m = 0; m <= c->M; ++m) {
      const uint32_t mf = level_first[m], mc = level_first[m + 1] - level_first[m];
      const uint32_t ng = (mc + gmax - 1) / gmax;
      for (uint32_t gi = 0; gi < ng; ++gi) {
        const uint32_t a = mf + (uint32_t)((uint64_t)mc * gi / ng);
        const uint32_t b = mf + (uint32_t)((uint64_t)mc * (gi + 1) / ng);
        for (const Row& r : rows) {
          if (D.woff[r.x + 1] == D.woff[r.x]) continue;
          const uint32_t it[kItemWords] = {(uint32_t)d, (uint32_t)m, a, b - a, r.x, r.c0, r.c1, 0};
          p.items.insert(p.items.end(), it, it + kItemWords);
        }
      }
    }
  }
}

struct Tables {
  std::vector<uint8_t> buf;
  size_t add(const void* src, size_t bytes) {
    const size_t o = align_up(buf.size(), 16);
    buf.resize(o + bytes);
    if (bytes) memcpy(buf.data() + o, src, bytes);
    return o;
  }
  size_t reserve(size_t bytes) {
    const size_t o = align_up(buf.size(), 16);
    buf.resize(o + bytes);
    return o;
  }
};

// Device memory for the plan; then serialise and upload the tables.
int plan_memory_and_tables(gakco_ctx* c, Plan& p, bool plain) {
  const uint64_t G = p.gtot;
  const uint64_t nm = c->masks.size();
  int rc;
#define ENSURE(buf, bytes)                                         \
  do {                                                             \
    if ((rc = ensure(c, c->buf, (size_t)(bytes), #buf)) != GAKCO_OK) return rc; \
  } while (0)
  ENSURE(fullkey, G * 8);
  ENSURE(win2seq, G * 4);
  const uint64_t pool = plain ? G : nm * G;
  ENSURE(ewin, pool * 4);
  ENSURE(eseq, pool * 4);
  ENSURE(efe, pool * 4);
  const uint64_t ce = p.max_chunk_elems;
  const size_t kbytes = p.any_wide ? 8 : 4;
  ENSURE(keyA, ce * kbytes);
  ENSURE(keyB, ce * kbytes);
  ENSURE(valA, ce * 4);
  ENSURE(valB, ce * 4);
  ENSURE(hist, p.max_hist * 4);
  ENSURE(tcnt, p.max_chunk_tiles * 8);
  ENSURE(segtot, p.max_chunk_nseg * 8);
  const uint64_t te = ce + p.max_chunk_nseg + 1;
  ENSURE(estart, te * 4);
  ENSURE(etseq, te * 4);
  ENSURE(efid, te * 4);
  ENSURE(fstart, te * 4);
  uint64_t nsum = 0;
  for (auto& D : p.ds) nsum += (uint64_t)D.n;
  ENSURE(rinv, nsum * 8);
  ENSURE(status, 128);
  if (plain) ENSURE(Cplain, (uint64_t)(c->M + 1) * p.nmax * p.nmax * 4);
  uint64_t csum = 0;
  for (auto& D : p.ds) csum += (uint64_t)(c->M + 1) * D.n * D.n;
  p.c_elems = csum;
  if (!plain) ENSURE(Cacc, csum * 4);

  Tables t;
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
  ENSURE(tables, t.buf.size());
  uint8_t* base = (uint8_t*)c->tables.p;
  double* rinv = (double*)c->rinv.p;
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
    rinv += D.n;
    in.C = plain ? nullptr : (uint32_t*)c->Cacc.p + cacc;
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
  p.ftiles = ftile;
  if (t.buf.size() > c->h_tables_cap) {
    if (c->h_tables) cudaFreeHost(c->h_tables);
    c->h_tables = nullptr;
    c->h_tables_cap = 0;
    size_t want = align_up(t.buf.size(), 1 << 16);
    cudaError_t e = cudaMallocHost(&c->h_tables, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->h_tables = nullptr;
      return fail(c, GAKCO_E_OOM, "cudaMallocHost(tables, %zu): %s", want, cudaGetErrorString(e));
    }
    c->h_tables_cap = want;
  }
  // The pinned staging area may still feed an earlier copy.
  cudaError_t e = cudaStreamSynchronize(c->cs);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream sync before table upload");
  memcpy(c->h_tables, t.buf.data(), t.buf.size());
  e = cudaMemcpyAsync(c->tables.p, c->h_tables, t.buf.size(), cudaMemcpyHostToDevice, c->cs);
  if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
#undef ENSURE
  return GAKCO_OK;
}

AccParams acc_params(gakco_ctx* c, const Plan& p, uint32_t* counter) {
  uint8_t* base = (uint8_t*)c->tables.p;
  AccParams a{};
  a.ds = (const DsInfo*)(base + p.o_info);
  a.items = (const uint32_t*)(base + p.o_items);
  a.nitems = (uint32_t)(p.items.size() / kItemWords);
  a.counter = counter;
  a.M = (uint32_t)c->M;
  a.gtot = p.gtot;
  a.ewin = (const uint32_t*)c->ewin.p;
  a.eseq = (const uint32_t*)c->eseq.p;
  a.efe = (const uint32_t*)c->efe.p;
  a.ncols = p.ncols;
  a.status = (uint32_t*)c->status.p;
  a.work = (unsigned long long*)((uint8_t*)c->status.p + 64);
  memcpy(a.h, c->h, sizeof a.h);
  memcpy(a.ie, c->ie, sizeof a.ie);
  return a;
}

// Sort and run-length pass over one chunk.
void enqueue_chunk(gakco_ctx* c, const Plan& p, const Chunk& ch) {
  uint8_t* base = (uint8_t*)c->tables.p;
  const SegDesc* segs = (const SegDesc*)(base + p.o_segs) + ch.seg_first;
  const uint32_t* tseg = (const uint32_t*)(base + p.o_tiles) + ch.tile_first;
  const MaskDesc* masks = (const MaskDesc*)(base + p.o_masks);
  void* kbuf[2] = {c->keyA.p, c->keyB.p};
  uint32_t* vbuf[2] = {(uint32_t*)c->valA.p, (uint32_t*)c->valB.p};
  void* kin = kbuf[1];  // the first pass extracts the masked keys here
  uint32_t* vin = nullptr;
  int cur = 0;
  for (size_t q = 0; q < ch.passes.size(); ++q) {
    Bracket b(c, "sort_pass", 3);
    launch_sort_pass(ch.wide, q == 0, segs, ch.nseg, tseg, ch.ntiles, masks,
                     (const uint64_t*)c->fullkey.p, kin, vin, kbuf[cur], vbuf[cur],
                     (uint32_t*)c->hist.p, ch.passes[q].first, ch.passes[q].second, c->cs);
    kin = kbuf[cur];
    vin = vbuf[cur];
    cur ^= 1;
  }
  Bracket b(c, "run_length", 4);
  launch_rle(ch.wide, segs, ch.nseg, tseg, ch.ntiles, kin, vin, (const uint32_t*)c->win2seq.p,
             (uint32_t*)c->tcnt.p, (uint32_t*)c->segtot.p, (uint32_t*)c->estart.p,
             (uint32_t*)c->etseq.p, (uint32_t*)c->efid.p, (uint32_t*)c->fstart.p,
             (uint32_t*)c->ewin.p, (uint32_t*)c->eseq.p, (uint32_t*)c->efe.p, c->cs);
}

// Everything after the table upload, on c->cs.
int enqueue_work(gakco_ctx* c, const Plan& p, bool plain) {
  uint8_t* base = (uint8_t*)c->tables.p;
  uint32_t* status = (uint32_t*)c->status.p;
  cudaMemsetAsync(status, 0, 128, c->cs);
  {
    Bracket b(c, "pack", 1);
    launch_pack((const DsPack*)(base + p.o_pack), (uint32_t)p.ds.size(), p.nseq, c->g, c->bits,
                c->sigma, (uint64_t*)c->fullkey.p, (uint32_t*)c->win2seq.p, status, c->cs);
  }
  if (!plain) {
    for (const Chunk& ch : p.chunks) enqueue_chunk(c, p, ch);
    AccParams a = acc_params(c, p, status + 8);
    if (p.c_elems) cudaMemsetAsync(c->Cacc.p, 0, p.c_elems * 4, c->cs);
    {
      Bracket b(c, "accumulate", 1);
      launch_accum(a, c->accum_threads, p.acc_blocks, p.acc_smem, c->cs);
    }
    {
      Bracket b(c, "diag", 1);
      launch_diag((const DsInfo*)(base + p.o_info), (uint32_t)p.ds.size(), p.nseq, a, c->cs);
    }
  } else {
    AccParams a = acc_params(c, p, status + 8);
    const DsInfo* infos = (const DsInfo*)(base + p.o_info);
    // Chunks are one segment each and ordered by level, then mask, then
    // dataset; handle one dataset at a time so C_m fits one buffer.
    for (size_t d = 0; d < p.ds.size(); ++d) {
      const DsHost& D = p.ds[d];
      if (D.n == 0) continue;
      const uint64_t nn = (uint64_t)D.n * D.n;
      cudaMemsetAsync(c->Cplain.p, 0, (size_t)(c->M + 1) * nn * 4, c->cs);
      for (const Chunk& ch : p.chunks) {
        if (p.seg_ds[ch.seg_first] != d) continue;
        const SegDesc& s = p.segs[ch.seg_first];
        enqueue_chunk(c, p, ch);
        Bracket b(c, "pairs_global", 1);
        launch_pairs_global((const uint32_t*)c->segtot.p, (const uint32_t*)c->eseq.p + s.pool,
                            (const uint32_t*)c->efe.p + s.pool, s.G,
                            (uint32_t*)c->Cplain.p + (uint64_t)ch.level * nn, (uint32_t)D.n,
                            status, c->cs);
      }
      Bracket b(c, "ie_combine", 1);
      launch_ie_combine(infos + d, (const uint32_t*)c->Cplain.p, (uint32_t)D.n, a, c->cs);
    }
  }
  if (plain) {
    Bracket b(c, "finish", 1);
    launch_finish((const DsInfo*)(base + p.o_info), (uint32_t)p.ds.size(), p.ftiles, (uint32_t)c->M,
                  p.want_nm, p.want_khat, c->cs);
  } else {
    Bracket b(c, "combine", 1);
    launch_combine((const DsInfo*)(base + p.o_info), (uint32_t)p.ds.size(), p.ftiles,
                   acc_params(c, p, status + 8), p.want_nm, p.want_khat, c->cs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return GAKCO_OK;
}

uint64_t plan_key(gakco_ctx* c, const Plan& p, bool plain) {
  uint64_t h = 1469598103934665603ull;
  int64_t o[8] = {plain, c->radix_bits, c->chunk_elems, c->accum_threads, c->smem_cols,
                  (int64_t)p.ds.size(), c->group_bytes, 0};
  h = fnv1a(h, o, sizeof o);
  for (const DsHost& D : p.ds) {
    const void* ptrs[4] = {D.codes, D.K, D.Khat, D.Nm};
    h = fnv1a(h, ptrs, sizeof ptrs);
    h = fnv1a(h, &D.n, sizeof D.n);
    if (D.n > 0) h = fnv1a(h, D.off, (D.n + 1) * 8);
  }
  return h;
}

int finish_call(gakco_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->status.p, 128, cudaMemcpyDeviceToHost, c->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->cs);
  if (e != cudaSuccess) return cuda_fail(c, e, "engine run");
  if (c->profile) {
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
  const uint32_t st = ((const uint32_t*)c->h_status)[0];
  const unsigned long long* wk = (const unsigned long long*)((const uint8_t*)c->h_status + 64);
  c->last_pairs = (double)wk[0];
  c->last_entries = (double)wk[1];
  c->last_windows = (double)wk[2];
  if (st & kErrBadCode) return fail(c, GAKCO_E_INVALID, "input holds a symbol >= sigma (%d)", c->sigma);
  if (st & kErrKneCM) return fail(c, GAKCO_E_INTERNAL, "internal check failed: sum h_m N_m != C_M");
  if (st & kErrBadEntry) return fail(c, GAKCO_E_INTERNAL, "internal check failed: entry out of range");
  if (st) return fail(c, GAKCO_E_INTERNAL, "device status 0x%x", st);
  return GAKCO_OK;
}

// The batched / plain engine on device buffers.
int run(gakco_ctx* c, Plan& p, cudaStream_t user) {
  const bool plain = c->engine == 1;
  c->launches = 0;
  c->timed.clear();
  c->ev_used = 0;
  c->last_replay = 0;
  c->last_mask_passes = 0;
  for (const DsHost& D : p.ds)
    if (D.G > 0) c->last_mask_passes += (int64_t)c->masks.size();
  if (p.ds.empty()) {
    c->last_launches = 0;
    return GAKCO_OK;
  }
  cudaError_t e = cudaEventRecord(c->ev_in, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cs, c->ev_in, 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream ordering");

  const bool graph = c->use_graph && !c->profile && !plain;
  const uint64_t key = graph ? plan_key(c, p, plain) : 0;
  int rc;
  if (graph && c->gexec && key == c->gkey) {
    // Same plan as the cached graph: tables and buffers are unchanged.
    e = cudaGraphLaunch(c->gexec, c->cs);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    c->launches = c->last_launches;
    c->last_replay = 1;
  } else {
    drop_graph(c);
    plan_chunks(c, p, plain);
    plan_items(c, p);
    if (!plain) {
      const int nb = accum_blocks_per_sm(c->accum_threads, p.acc_smem);
      if (nb <= 0)
        return fail(c, GAKCO_E_CUDA, "accumulation kernel does not fit (%zu B shared)", p.acc_smem);
      p.acc_blocks = nb * c->nsm;
    }
    if ((rc = plan_memory_and_tables(c, p, plain)) != GAKCO_OK) return rc;
    if (graph) {
      cudaGraph_t gr = nullptr;
      e = cudaStreamBeginCapture(c->cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
      rc = enqueue_work(c, p, plain);
      e = cudaStreamEndCapture(c->cs, &gr);
      if (rc != GAKCO_OK) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
      e = cudaGraphInstantiate(&c->gexec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, e, "graph instantiate");
      }
      c->gkey = key;
      e = cudaGraphLaunch(c->gexec, c->cs);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    } else {
      if ((rc = enqueue_work(c, p, plain)) != GAKCO_OK) return rc;
    }
  }
  c->last_launches = c->launches;
  rc = finish_call(c);
  e = cudaEventRecord(c->ev_out, c->cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, c->ev_out, 0);
  if (e != cudaSuccess && rc == GAKCO_OK) rc = cuda_fail(c, e, "stream ordering");
  return rc;
}

int gram_host(gakco_ctx* c, int32_t nd, const uint8_t* const* codes, const int64_t* const* off,
              const int32_t* n, int32_t* const* K, double* const* Khat, int32_t* const* Nm) {
  Plan p;
  int rc = plan_datasets(c, p, nd, codes, off, n, K, Khat, Nm, false);
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
  if ((rc = ensure(c, c->codes, cbytes + 16, "codes")) != GAKCO_OK) return rc;
  if ((rc = ensure(c, c->outK, kel * 4 + 16, "K")) != GAKCO_OK) return rc;
  if (want_khat && (rc = ensure(c, c->outKhat, kel * 8 + 16, "Khat")) != GAKCO_OK) return rc;
  if (want_nm && (rc = ensure(c, c->outNm, nmel * 4 + 16, "Nm")) != GAKCO_OK) return rc;
  cudaError_t e = cudaSuccess;
  for (int32_t d = 0; d < nd && e == cudaSuccess; ++d) {
    DsHost& D = p.ds[d];
    const uint8_t* dc = (const uint8_t*)c->codes.p + coff[d];
    if (D.n > 0 && D.off[D.n] > 0)
      e = cudaMemcpyAsync((void*)dc, D.codes, (size_t)D.off[D.n], cudaMemcpyHostToDevice, c->cs);
    D.codes = dc;
    D.K = (int32_t*)c->outK.p + koff[d];
    D.Khat = D.Khat ? (double*)c->outKhat.p + koff[d] : nullptr;
    D.Nm = D.Nm ? (int32_t*)c->outNm.p + nmoff[d] : nullptr;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "copy codes to device");
  rc = run(c, p, c->cs);
  if (rc != GAKCO_OK) return rc;
  for (int32_t d = 0; d < nd && e == cudaSuccess; ++d) {
    const DsHost& D = p.ds[d];
    const size_t nn = (size_t)D.n * D.n;
    if (K && K[d] && nn) e = cudaMemcpyAsync(K[d], D.K, nn * 4, cudaMemcpyDeviceToHost, c->cs);
    if (e == cudaSuccess && Khat && Khat[d] && nn)
      e = cudaMemcpyAsync(Khat[d], D.Khat, nn * 8, cudaMemcpyDeviceToHost, c->cs);
    if (e == cudaSuccess && Nm && Nm[d] && nn)
      e = cudaMemcpyAsync(Nm[d], D.Nm, (size_t)(c->M + 1) * nn * 4, cudaMemcpyDeviceToHost, c->cs);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->cs);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy results to host");
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
      md.kbits = (uint32_t)((g - m) * bits);
      const int nk = (int)keep.size();
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
    c->h[m] = (uint32_t)binom(g - m, k);                       // Eq. 6
    for (int j = 0; j < m; ++j) c->ie[m][j] = (uint32_t)binom(g - j, m - j);  // Eq. 9
    c->maxC = std::max<uint32_t>(c->maxC, (uint32_t)binom(g, m));
  }

  cudaError_t e = cudaGetDevice(&c->device);
  int v = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->smem_optin = (size_t)v;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, 128);
  if (e == cudaSuccess) e = (cudaError_t)prep_init();
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
  if (c->cs) cudaStreamSynchronize(c->cs);
  drop_graph(c);
  DevBuf* bufs[] = {&c->fullkey, &c->win2seq, &c->ewin, &c->eseq, &c->efe, &c->keyA,
                    &c->keyB,    &c->valA,    &c->valB, &c->hist, &c->tcnt, &c->segtot,
                    &c->estart,  &c->etseq,   &c->efid, &c->fstart, &c->tables, &c->codes,
                    &c->outK,    &c->outKhat, &c->outNm, &c->rinv, &c->status, &c->Cplain,
                    &c->Cacc};
  for (DevBuf* b : bufs) release(*b);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->h_tables) cudaFreeHost(c->h_tables);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->cs) cudaStreamDestroy(c->cs);
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
    case GAKCO_OPT_GROUP_BYTES:
      if (v < 1) return fail(c, GAKCO_E_INVALID, "group bytes must be >= 1");
      c->group_bytes = v;
      break;
    case GAKCO_OPT_FAIL_ALLOC_AFTER:
      if (v < 0) return fail(c, GAKCO_E_INVALID, "allocation countdown must be >= 0");
      c->fail_alloc_after = v;
      break;
    default:
      return fail(c, GAKCO_E_INVALID, "unknown option %d", key);
  }
  drop_graph(c);
  return GAKCO_OK;
}

int gakco_get_stat(const gakco_ctx* c, int key, double* v) {
  if (!c || !v) return GAKCO_E_INVALID;
  switch (key) {
    case GAKCO_STAT_LAUNCHES:
      *v = (double)c->last_launches;
      return GAKCO_OK;
    case GAKCO_STAT_MASK_PASSES:
      *v = (double)c->last_mask_passes;
      return GAKCO_OK;
    case GAKCO_STAT_DEVICE_BYTES: {
      const DevBuf* bufs[] = {&c->fullkey, &c->win2seq, &c->ewin, &c->eseq, &c->efe, &c->keyA,
                              &c->keyB,    &c->valA,    &c->valB, &c->hist, &c->tcnt, &c->segtot,
                              &c->estart,  &c->etseq,   &c->efid, &c->fstart, &c->tables, &c->codes,
                              &c->outK,    &c->outKhat, &c->outNm, &c->rinv, &c->status, &c->Cplain,
                              &c->Cacc};
      double s = 0;
      for (const DevBuf* b : bufs) s += (double)b->cap;
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
  return gram_host(c, 1, &codes, &offsets, &n, &K, &Khat, &Nm);
}

int gakco_gram_batch(gakco_ctx* c, int32_t nd, const uint8_t* const* codes,
                     const int64_t* const* offsets, const int32_t* n, int32_t* const* K,
                     double* const* Khat, int32_t* const* Nm) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  return gram_host(c, nd, codes, offsets, n, K, Khat, Nm);
}

int gakco_gram_batch_device(gakco_ctx* c, int32_t nd, const uint8_t* const* codes,
                            const int64_t* const* offsets, const int32_t* n, int32_t* const* K,
                            double* const* Khat, int32_t* const* Nm, void* stream) {
  if (!c) return GAKCO_E_INVALID;
  c->err.clear();
  Plan p;
  int rc = plan_datasets(c, p, nd, codes, offsets, n, K, Khat, Nm, true);
  if (rc != GAKCO_OK) return rc;
  return run(c, p, (cudaStream_t)stream);
}

int gakco_gram_device(gakco_ctx* c, const uint8_t* codes, const int64_t* offsets, int32_t n,
                      int32_t* K, double* Khat, int32_t* Nm, void* stream) {
  return gakco_gram_batch_device(c, 1, &codes, &offsets, &n, &K, &Khat, &Nm, stream);
}

}  // extern "C"
