// Out-of-core sparse A-passes (Section 3.5 in-core / out-of-core switching,
// Section 3.7 I/O overlapped with compute) for a CSR matrix held in host
// memory, over the block-cyclic tiles of Section 3.1 (blocks as ranges of row
// and column indices) in the sparse storage of Section 3.3.
//
// The forward pass Y = A X visits the tiles of the CSR of A, the transposed
// pass Z = A^T Y those of the CSR of A^T: tile (I, J) of an orientation holds
// the entries in rows [I mb, ...) and columns [J nb, ...) of that matrix, as a
// CSR with row offsets starting at 0 and column indices relative to the tile's
// first column.  Full-width tiles (the default) are plain ranges of the host
// arrays and are copied as they are (the row offsets rebased on the device);
// narrower tiles are cut from the host CSR once per run into a pinned host
// store.  Tile t goes to device slot t mod S and is copied on a side stream
// while the tile before it is multiplied; the compute stream waits for the
// copy's event, and the next copy into a slot waits for the product that read
// it.  Tiles that fit in the memory left under the cap stay resident after
// their first copy of a run.  Each output row block is written by its tiles in
// tile order (added when the columns are tiled), so the result does not depend
// on timing.
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

rsvd_status csr_tile_host(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx, const float* val,
                          int64_t row0, int64_t row1, int64_t col0, int64_t col1, int32_t* t_rowptr,
                          int32_t* t_colidx, float* t_val, int64_t cap, int64_t* nnz_out) {
  if (m < 0 || n < 0 || !rowptr || !nnz_out || row0 < 0 || row1 < row0 || row1 > m || col0 < 0 || col1 < col0 ||
      col1 > n || cap < 0)
    return fail(RSVD_ERR_INVALID_ARG, "csr_tile: bad arguments");
  if (cap > 0 && (!t_colidx || !t_val))
    return fail(RSVD_ERR_INVALID_ARG, "csr_tile: NULL output arrays with cap > 0");
  int64_t cnt = 0;
  if (t_rowptr) t_rowptr[0] = 0;
  for (int64_t i = row0; i < row1; ++i) {
    const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
    if (e1 < e0) return fail(RSVD_ERR_INVALID_ARG, "csr_tile: rowptr decreases");
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t c = colidx[e];
      if (c < col0 || c >= col1) continue;
      if (cnt < cap) {
        t_colidx[cnt] = (int32_t)(c - col0);
        t_val[cnt] = val[e];
      }
      ++cnt;
    }
    if (t_rowptr) {
      if (cnt > 0x7fffffffLL) return fail(RSVD_ERR_INVALID_ARG, "csr_tile: more than 2^31 - 1 entries");
      t_rowptr[i - row0 + 1] = (int32_t)cnt;
    }
  }
  *nnz_out = cnt;
  if (cap > 0 && cnt > cap) return fail(RSVD_ERR_INVALID_ARG, "csr_tile: cap below the tile's entry count");
  return RSVD_OK;
}

namespace {

__global__ void rebase_kernel(int32_t* __restrict__ rp, int64_t count, int32_t base) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    rp[i] -= base;
}

struct CsrTile {
  int64_t row0 = 0, rows = 0, col0 = 0, cols = 0, nnz = 0;
  const int32_t* rp = nullptr;  // host: rows + 1 offsets (minus `base` gives the tile's own)
  const int32_t* ci = nullptr;  // host: nnz column indices (relative to col0)
  const float* v = nullptr;     // host: nnz values
  int32_t base = 0;
  size_t bytes() const { return (size_t)(rows + 1) * 4 + (size_t)nnz * 8; }
};

}  // namespace

struct CsrOrient {
  int64_t M = 0, K = 0, mb = 0, nb = 0;
  bool col_tiled = false;
  std::vector<CsrTile> tiles;
  // narrow tiles: their CSRs cut into one pinned host buffer
  char* store = nullptr;
  size_t store_bytes = 0;
  std::vector<void*> cache;
  std::vector<char> cache_valid;
  std::vector<cudaEvent_t> cache_ev;
  ~CsrOrient() {
    for (void* p : cache) cudaFree(p);
    for (auto e : cache_ev) cudaEventDestroy(e);
    if (store) cudaFreeHost(store);
  }
};

struct CsrStream {
  int S = 2;
  size_t slot_bytes = 0;
  std::vector<void*> slot;
  std::vector<cudaEvent_t> copied, freed;
  cudaStream_t copy = nullptr;
  CsrOrient o[2];              // 0: tiles of the CSR of A, 1: tiles of the CSR of A^T
  void* sws = nullptr;         // SpMM long-row workspace (largest tile)
  size_t sws_bytes = 0;
  uint64_t h2d_bytes = 0;
  int64_t tiles_per_pass = 0, tiles_cached = 0;
  ~CsrStream() {
    for (void* p : slot) cudaFree(p);
    for (auto e : copied) cudaEventDestroy(e);
    for (auto e : freed) cudaEventDestroy(e);
    if (copy) cudaStreamDestroy(copy);
    if (sws) cudaFree(sws);
  }
};

void csr_stream_free(CsrStream* s) { delete s; }

void csr_stream_stats(const CsrStream* s, uint64_t* h2d, int64_t* per_pass, int64_t* cached) {
  if (h2d) *h2d = s ? s->h2d_bytes : 0;
  if (per_pass) *per_pass = s ? s->tiles_per_pass : 0;
  if (cached) *cached = s ? s->tiles_cached : 0;
}

namespace {

CsrTile row_range_tile(const int32_t* rp, const int32_t* ci, const float* v, int64_t K, int64_t row0,
                       int64_t rows) {
  CsrTile t;
  t.row0 = row0;
  t.rows = rows;
  t.col0 = 0;
  t.cols = K;
  t.base = rp[row0];
  t.nnz = (int64_t)rp[row0 + rows] - t.base;
  t.rp = rp + row0;
  t.ci = ci + t.base;
  t.v = v + t.base;
  return t;
}

// Default tiles of one orientation: full-width row ranges cut where the entry
// count would pass `target` (a row longer than that is a tile of its own), so
// that skewed row lengths give tiles of similar size.
void build_balanced_tiles(CsrOrient& o, int64_t M, int64_t K, const int32_t* rp, const int32_t* ci, const float* v,
                          int64_t target) {
  o.M = M; o.K = K; o.mb = 0; o.nb = K;
  o.col_tiled = false;
  o.tiles.clear();
  int64_t row0 = 0;
  while (row0 < M) {
    int64_t row1 = row0 + 1;
    // the last row r with rp[r] - rp[row0] <= target, at least one row
    const int64_t limit = (int64_t)rp[row0] + target;
    const int32_t* it = std::upper_bound(rp + row0 + 1, rp + M + 1, (int32_t)std::min<int64_t>(limit, 0x7fffffffLL));
    const int64_t cand = (int64_t)(it - rp) - 1;
    if (cand > row1) row1 = cand;
    o.tiles.push_back(row_range_tile(rp, ci, v, K, row0, row1 - row0));
    row0 = row1;
  }
}

// Tiles of one orientation (an M x K CSR) on the block-cyclic grid mb x nb.
// Full-width tiles point into the host arrays; narrower ones are cut into
// o.store.
rsvd_status build_tiles(CsrOrient& o, int64_t M, int64_t K, const int32_t* rp, const int32_t* ci, const float* v,
                        int64_t mb, int64_t nb) {
  o.M = M; o.K = K; o.mb = mb; o.nb = nb;
  o.col_tiled = nb < K;
  o.tiles.clear();
  const int64_t Tm = cdiv(M, mb), Tn = cdiv(K, nb);
  if (!o.col_tiled) {
    for (int64_t I = 0; I < Tm; ++I) o.tiles.push_back(row_range_tile(rp, ci, v, K, I * mb, std::min(mb, M - I * mb)));
    return RSVD_OK;
  }
  // count every tile's entries (threads over tile rows), then cut them
  std::vector<int64_t> cnt((size_t)(Tm * Tn), 0);
  std::vector<char> bad((size_t)Tm, 0);
  auto count_row = [&](int64_t I) {
    const int64_t r0 = I * mb, r1 = std::min(M, r0 + mb);
    for (int64_t i = r0; i < r1; ++i)
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int64_t c = ci[e];
        if (c < 0 || c >= K) { bad[(size_t)I] = 1; return; }
        ++cnt[(size_t)(I * Tn + c / nb)];
      }
  };
  unsigned hw = std::thread::hardware_concurrency();
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 32, Tm}));
  auto run_rows = [&](auto fn) {
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t)
      th.emplace_back([&, t] { for (int64_t I = t; I < Tm; I += T) fn(I); });
    for (int64_t I = 0; I < Tm; I += T) fn(I);
    for (auto& x : th) x.join();
  };
  run_rows(count_row);
  for (char b : bad)
    if (b) return fail(RSVD_ERR_INVALID_ARG, "CSR streaming: column index out of range");
  size_t total = 0;
  std::vector<size_t> off((size_t)(Tm * Tn));
  for (int64_t t = 0; t < Tm * Tn; ++t) {
    const int64_t I = t / Tn;
    const int64_t rows = std::min(mb, M - I * mb);
    off[(size_t)t] = total;
    total += round_up((size_t)(rows + 1) * 4, 16) + round_up((size_t)cnt[(size_t)t] * 4, 16) * 2;
  }
  if (o.store_bytes < total) {
    if (o.store) cudaFreeHost(o.store);
    o.store = nullptr;
    o.store_bytes = 0;
    RSVD_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&o.store), total, cudaHostAllocDefault));
    o.store_bytes = total;
  }
  o.tiles.resize((size_t)(Tm * Tn));
  for (int64_t t = 0; t < Tm * Tn; ++t) {
    const int64_t I = t / Tn, J = t % Tn;
    CsrTile& x = o.tiles[(size_t)t];
    x.row0 = I * mb;
    x.rows = std::min(mb, M - x.row0);
    x.col0 = J * nb;
    x.cols = std::min(nb, K - x.col0);
    x.nnz = cnt[(size_t)t];
    x.base = 0;
    char* p = o.store + off[(size_t)t];
    x.rp = reinterpret_cast<const int32_t*>(p);
    p += round_up((size_t)(x.rows + 1) * 4, 16);
    x.ci = reinterpret_cast<const int32_t*>(p);
    p += round_up((size_t)x.nnz * 4, 16);
    x.v = reinterpret_cast<const float*>(p);
  }
  std::vector<rsvd_status> st((size_t)Tm, RSVD_OK);
  auto cut_row = [&](int64_t I) {
    for (int64_t J = 0; J < Tn; ++J) {
      CsrTile& x = o.tiles[(size_t)(I * Tn + J)];
      int64_t got = 0;
      const rsvd_status s = csr_tile_host(M, K, rp, ci, v, x.row0, x.row0 + x.rows, x.col0, x.col0 + x.cols,
                                          const_cast<int32_t*>(x.rp), const_cast<int32_t*>(x.ci),
                                          const_cast<float*>(x.v), x.nnz, &got);
      if (s != RSVD_OK || got != x.nnz) st[(size_t)I] = RSVD_ERR_INVALID_ARG;
    }
  };
  run_rows(cut_row);
  for (auto s : st)
    if (s != RSVD_OK) return fail(RSVD_ERR_INVALID_ARG, "CSR streaming: tile cutting failed");
  return RSVD_OK;
}

}  // namespace

rsvd_status csr_stream_prepare(CsrStream** ps, const rsvd_matrix& A, int64_t mb_req, int64_t nb_req, int slots,
                               size_t budget, int r) {
  if (slots < 1) slots = 2;
  const int64_t m = A.m, n = A.n, nnz = A.nnz;
  delete *ps;
  CsrStream* s = new CsrStream();
  *ps = s;
  s->S = slots;
  // tile edges: the options' mb x nb for A (and nb x mb for A^T, the same
  // blocks transposed); by default full-width row ranges of at most 32 Mi
  // entries, the target halved until S slots and the workspace take at most
  // half of the budget
  const bool grid = mb_req > 0 || nb_req > 0;
  int64_t target = std::max<int64_t>(1, std::min<int64_t>((int64_t)1 << 25, nnz / 8 + 1));
  for (int attempt = 0; attempt < 40; ++attempt) {
    if (grid) {
      const int64_t mbA = mb_req > 0 ? std::min(mb_req, m) : m;
      const int64_t nbA = nb_req > 0 ? std::min(nb_req, n) : n;
      RSVD_TRY(build_tiles(s->o[0], m, n, A.rowptr, A.colidx, A.val, mbA, nbA));
      RSVD_TRY(build_tiles(s->o[1], n, m, A.t_rowptr, A.t_colidx, A.t_val, nbA, mbA));
    } else {
      build_balanced_tiles(s->o[0], m, n, A.rowptr, A.colidx, A.val, target);
      build_balanced_tiles(s->o[1], n, m, A.t_rowptr, A.t_colidx, A.t_val, target);
    }
    size_t biggest = 0;
    int64_t max_nnz = 0;
    for (auto& o : s->o)
      for (auto& t : o.tiles) {
        biggest = std::max(biggest, t.bytes());
        max_nnz = std::max(max_nnz, t.nnz);
      }
    s->slot_bytes = round_up(biggest, 256) + 512;
    s->sws_bytes = spmm_ws_bytes(max_nnz, r);
    const size_t fixed = (size_t)slots * s->slot_bytes + s->sws_bytes;
    if (fixed <= budget / 2 || (grid && fixed <= budget)) break;
    if (grid || target <= 4096) return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_run: mem_cap leaves no room for the CSR tiles");
    target /= 2;
  }
  const size_t fixed = (size_t)slots * s->slot_bytes + s->sws_bytes;
  if (fixed > budget) return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_run: mem_cap leaves no room for the CSR tiles");
  RSVD_CUDA(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking));
  RSVD_CUDA(cudaMalloc(&s->sws, s->sws_bytes));
  for (int i = 0; i < slots; ++i) {
    void* p = nullptr;
    RSVD_CUDA(cudaMalloc(&p, s->slot_bytes));
    s->slot.push_back(p);
    cudaEvent_t a, b;
    RSVD_CUDA(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    RSVD_CUDA(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    s->copied.push_back(a);
    s->freed.push_back(b);
  }
  // resident cache: the rest of the budget, half per orientation, tiles in
  // visit order
  size_t left = budget - fixed;
  int64_t total_tiles = 0;
  for (int k = 0; k < 2; ++k) {
    CsrOrient& o = s->o[k];
    size_t share = k == 0 ? left / 2 : left;
    for (auto& t : o.tiles) {
      const size_t b = round_up(t.bytes(), 256) + 512;
      if (b > share) break;
      void* p = nullptr;
      if (cudaMalloc(&p, b) != cudaSuccess) {
        (void)cudaGetLastError();
        break;
      }
      o.cache.push_back(p);
      cudaEvent_t e;
      RSVD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      o.cache_ev.push_back(e);
      share -= b;
      left -= b;
    }
    o.cache_valid.assign(o.cache.size(), 0);
    s->tiles_cached += (int64_t)o.cache.size();
    total_tiles += (int64_t)o.tiles.size();
  }
  s->tiles_per_pass = total_tiles - s->tiles_cached;
  return RSVD_OK;
}

void csr_stream_begin_run(CsrStream* s) {
  s->h2d_bytes = 0;
  for (auto& o : s->o) std::fill(o.cache_valid.begin(), o.cache_valid.end(), 0);
}

rsvd_status csr_apass_streamed(CsrStream* s, int trans, int r, const SpmmPanel& X, float* Y, int64_t ldy,
                               cudaStream_t st) {
  CsrOrient& o = s->o[trans ? 1 : 0];
  if (o.col_tiled) RSVD_CUDA(cudaMemsetAsync(Y, 0, (size_t)o.M * ldy * sizeof(float), st));
  for (size_t t = 0; t < o.tiles.size(); ++t) {
    const CsrTile& T = o.tiles[t];
    const bool cached = t < o.cache.size();
    const int slot = (int)(t % (size_t)s->S);
    char* dev = static_cast<char*>(cached ? o.cache[t] : s->slot[slot]);
    int32_t* d_rp = reinterpret_cast<int32_t*>(dev);
    int32_t* d_ci = reinterpret_cast<int32_t*>(dev + round_up((size_t)(T.rows + 1) * 4, 256));
    float* d_v = reinterpret_cast<float*>(reinterpret_cast<char*>(d_ci) + round_up((size_t)T.nnz * 4, 256));
    if (!cached || !o.cache_valid[t]) {
      if (!cached) RSVD_CUDA(cudaStreamWaitEvent(s->copy, s->freed[slot], 0));
      RSVD_CUDA(cudaMemcpyAsync(d_rp, T.rp, (size_t)(T.rows + 1) * 4, cudaMemcpyHostToDevice, s->copy));
      if (T.nnz) {
        RSVD_CUDA(cudaMemcpyAsync(d_ci, T.ci, (size_t)T.nnz * 4, cudaMemcpyHostToDevice, s->copy));
        RSVD_CUDA(cudaMemcpyAsync(d_v, T.v, (size_t)T.nnz * 4, cudaMemcpyHostToDevice, s->copy));
      }
      if (T.base) {
        const int blocks = (int)std::min<int64_t>(cdiv(T.rows + 1, 256), 1024);
        rebase_kernel<<<blocks, 256, 0, s->copy>>>(d_rp, T.rows + 1, T.base);
        RSVD_CUDA(after_launch());
      }
      cudaEvent_t done = cached ? o.cache_ev[t] : s->copied[slot];
      RSVD_CUDA(cudaEventRecord(done, s->copy));
      RSVD_CUDA(cudaStreamWaitEvent(st, done, 0));
      s->h2d_bytes += T.bytes();
      if (cached) o.cache_valid[t] = 1;
    }
    SpmmPanel xt = X;  // the panel rows of the tile's columns
    if (xt.f) xt.f += T.col0 * xt.ld;
    if (xt.h) xt.h += T.col0 * xt.ld;
    if (xt.p24) xt.p24 += T.col0 * xt.rb;
    RSVD_TRY(spmm_csr_panel(T.rows, r, d_rp, d_ci, d_v, T.nnz, xt, Y + T.row0 * ldy, ldy, o.col_tiled, s->sws,
                            s->sws_bytes, st));
    if (!cached) RSVD_CUDA(cudaEventRecord(s->freed[slot], st));
  }
  return RSVD_OK;
}

}  // namespace rsvd
