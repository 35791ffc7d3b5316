// Out-of-core A-passes (Section 3.5 in-core / out-of-core switching, Section
// 3.7 I/O overlapped with compute) for a dense A held in pinned host memory.
//
// The tiles of the block-cyclic map (Section 3.1) are visited in order
// t = I*Tn + J.  Tile t is copied with cudaMemcpy2DAsync on a side stream into
// device slot t mod S (S slots: double buffering for S = 2), the compute
// stream waits for that copy's event, multiplies the tile into the panel
// (Y[I] += A[I,J] X[J] forward, Z[J] += A[I,J]^T Y[I] transposed, in tile
// order, so the sums do not depend on timing), and records the slot's "free"
// event that the next copy into the slot waits for.  Tiles that fit in the
// device memory left under the cap after the workspace and the slots stay
// resident after their first copy of a run (the resident cache), so later
// passes of the same run stream only the rest.  BF16 plans keep the cached
// tiles as their BF16 copy instead (half the bytes, so twice the tiles under
// the same cap): the first forward pass of a run streams each such tile in
// FP32 and writes its BF16 copy while multiplying it (the same operands, so the
// same products), the later BF16 passes read the copy, and a pass in another
// precision (the split-BF16 B^T, which needs FP32 A) streams the tile again.
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

struct StreamState {
  int S = 2;
  int64_t mb = 0, nb = 0, ld_tile = 0;
  size_t tile_bytes = 0;
  std::vector<void*> slot;
  std::vector<void*> cache;          // resident copies of tiles 0 .. ncache-1
  bool cache16 = false;              // the cache holds BF16 copies (row stride ld16)
  int64_t ld16 = 0;
  std::vector<char> cache_valid;     // filled during the current run
  std::vector<cudaEvent_t> copied;   // per slot
  std::vector<cudaEvent_t> freed;    // per slot
  std::vector<cudaEvent_t> cache_ev; // per cached tile
  cudaStream_t copy = nullptr;
  uint64_t h2d_bytes = 0;            // copied during the last run
  int64_t tiles_per_pass = 0, tiles_cached = 0;
  size_t device_bytes = 0;
  void* ws = nullptr;                // A-pass workspace sized for one tile
  size_t ws_bytes = 0;
  void* ytile = nullptr;             // fused sweeps: A_I W of the current row panel (mb x ldr)
  size_t ytile_bytes = 0;

  ~StreamState() {
    for (void* p : slot) cudaFree(p);
    for (void* p : cache) cudaFree(p);
    for (auto e : copied) cudaEventDestroy(e);
    for (auto e : freed) cudaEventDestroy(e);
    for (auto e : cache_ev) cudaEventDestroy(e);
    if (copy) cudaStreamDestroy(copy);
    if (ws) cudaFree(ws);
    if (ytile) cudaFree(ytile);
  }
};

void stream_state_free(StreamState* s) { delete s; }

static int slot_of(const StreamState* s, int64_t t) { return (int)(t % s->S); }

void stream_stats(const StreamState* s, uint64_t* h2d, int64_t* per_pass, int64_t* cached) {
  if (h2d) *h2d = s ? s->h2d_bytes : 0;
  if (per_pass) *per_pass = s ? s->tiles_per_pass : 0;
  if (cached) *cached = s ? s->tiles_cached : 0;
}

// Build (or reuse) the streaming state for an m x n host matrix of element
// size esz within `budget` device bytes (the cap minus the plan workspace).
rsvd_status stream_prepare(StreamState** ps, int64_t m, int64_t n, size_t esz, int64_t mb_req, int64_t nb_req,
                           int slots, size_t budget, int r, int prec, int final_prec, bool bf16_cache) {
  if (slots < 1) slots = 2;
  // Default tile: a full-width row panel of about 512 MB (or less, to leave room
  // for the resident cache).  Rows of a panel are contiguous in host memory, and
  // a contiguous copy runs at the full pinned host-to-device rate, while pitched
  // copies of narrow tiles (tens of KB per row) reach about half of it.
  int64_t nb = nb_req > 0 ? nb_req : n;
  int64_t mb = mb_req;
  if (mb <= 0) {
    const size_t target = (size_t)512 << 20;
    const size_t per_row = (size_t)round_up(nb, 4) * esz;
    mb = (int64_t)(target / per_row);
    const size_t share = budget / (size_t)(slots + 2);
    if ((size_t)mb * per_row > share) mb = (int64_t)(share / per_row);
    if (mb < 16) mb = 16;
  }
  if (mb > m) mb = m;
  if (nb > n) nb = n;
  // shrink the tiles until the slots fit the budget
  while ((size_t)slots * mb * round_up(nb, 4) * esz > budget && (mb > 16 || nb > 16)) {
    if (mb >= nb && mb > 16) mb = (mb + 1) / 2;
    else if (nb > 16) nb = (nb + 1) / 2;
  }
  const int64_t ld_tile = round_up(nb, 4);
  const size_t tile_bytes = (size_t)mb * ld_tile * esz;
  // A-pass workspace for every tile shape (full, last tile row/column, corner)
  size_t tws = 0;
  const int64_t rows_opts[2] = {mb, m % mb ? m % mb : mb};
  const int64_t cols_opts[2] = {nb, n % nb ? n % nb : nb};
  for (int64_t tr_rows : rows_opts)
    for (int64_t tr_cols : cols_opts)
      for (int tr = 0; tr < 2; ++tr)
        for (int pr : {prec, final_prec, sweep_trans_prec(prec)}) {
          const size_t b = apass_ws_bytes(tr_rows, tr_cols, r, tr, pr, 0, 0) + 512;
          if (b > tws) tws = b;
        }
  // fused sweeps keep A_I W of one row panel (FP32 or FP64, ldr columns)
  const size_t ytile_bytes = (size_t)mb * round_up(r, 4) * (esz == 8 ? 8 : 4) + 256;
  if ((size_t)slots * tile_bytes + tws + ytile_bytes > budget)
    return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_run: mem_cap leaves no room for the streaming slots");
  StreamState* s = *ps;
  if (s && s->mb == mb && s->nb == nb && s->S == slots && s->tile_bytes == tile_bytes && s->cache16 == bf16_cache)
    return RSVD_OK;
  delete s;
  s = new StreamState();
  *ps = s;
  s->S = slots;
  s->mb = mb;
  s->nb = nb;
  s->ld_tile = ld_tile;
  s->tile_bytes = tile_bytes;
  s->cache16 = bf16_cache;
  s->ld16 = round_up(nb, 64);
  RSVD_CUDA(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking));
  RSVD_CUDA(cudaMalloc(&s->ws, tws));
  s->ws_bytes = tws;
  RSVD_CUDA(cudaMalloc(&s->ytile, ytile_bytes));
  s->ytile_bytes = ytile_bytes;
  for (int i = 0; i < slots; ++i) {
    void* p = nullptr;
    RSVD_CUDA(cudaMalloc(&p, tile_bytes));
    s->slot.push_back(p);
    cudaEvent_t a, b;
    RSVD_CUDA(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    RSVD_CUDA(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    s->copied.push_back(a);
    s->freed.push_back(b);
  }
  const int64_t ntiles = cdiv(m, mb) * cdiv(n, nb);
  const size_t cache_tile_bytes = bf16_cache ? (size_t)mb * s->ld16 * 2 : tile_bytes;
  int64_t ncache = (int64_t)((budget - (size_t)slots * tile_bytes - tws - ytile_bytes) / cache_tile_bytes);
  if (ncache > ntiles) ncache = ntiles;
  for (int64_t t = 0; t < ncache; ++t) {
    void* p = nullptr;
    if (cudaMalloc(&p, cache_tile_bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      break;
    }
    s->cache.push_back(p);
    cudaEvent_t e;
    RSVD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    s->cache_ev.push_back(e);
  }
  s->cache_valid.assign(s->cache.size(), 0);
  s->tiles_cached = (int64_t)s->cache.size();
  s->tiles_per_pass = ntiles - s->tiles_cached;
  s->device_bytes = (size_t)slots * tile_bytes + s->cache.size() * cache_tile_bytes + tws + ytile_bytes;
  return RSVD_OK;
}

void stream_begin_run(StreamState* s) {
  s->h2d_bytes = 0;
  std::fill(s->cache_valid.begin(), s->cache_valid.end(), 0);
}

namespace {

// Make tile t (rows [row0, row0+rows) x cols [col0, col0+cols)) available on
// the device for the compute stream: a resident copy, or a copy into its slot
// on the side stream that the compute stream waits for.  Returns the device
// tile (row stride ld_tile) and whether it is resident.
rsvd_status fetch_tile(StreamState* s, const rsvd_matrix& Ah, int64_t t, int64_t row0, int64_t col0, int64_t rows,
                       int64_t cols, size_t esz, cudaStream_t st, rsvd_matrix* T, bool* cached_out) {
  // a BF16 cache holds no FP32 tiles: the FP32 tile goes through a slot
  const bool cached = !s->cache16 && t < (int64_t)s->cache.size();
  const int slot = (int)(t % s->S);
  void* tile = cached ? s->cache[t] : s->slot[slot];
  if (!cached || !s->cache_valid[t]) {
    const char* host = static_cast<const char*>(Ah.data);
    if (!cached) RSVD_CUDA(cudaStreamWaitEvent(s->copy, s->freed[slot], 0));
    RSVD_CUDA(cudaMemcpy2DAsync(tile, (size_t)s->ld_tile * esz, host + ((size_t)row0 * Ah.ld + col0) * esz,
                                (size_t)Ah.ld * esz, (size_t)cols * esz, (size_t)rows, cudaMemcpyHostToDevice,
                                s->copy));
    cudaEvent_t done = cached ? s->cache_ev[t] : s->copied[slot];
    RSVD_CUDA(cudaEventRecord(done, s->copy));
    RSVD_CUDA(cudaStreamWaitEvent(st, done, 0));
    s->h2d_bytes += (uint64_t)rows * cols * esz;
    if (cached) s->cache_valid[t] = 1;
  }
  *T = Ah;
  T->location = RSVD_ON_DEVICE;
  T->m = rows;
  T->n = cols;
  T->data = tile;
  T->ld = s->ld_tile;
  *cached_out = cached;
  return RSVD_OK;
}

}  // namespace

int sweep_trans_prec(int prec) { return prec == RSVD_PREC_BF16 ? RSVD_PREC_BF16X3 : prec; }

// One streamed A-pass.  X: K x r panel (K = n forward, m transposed), Y: M x r
// output, both device, leading dimension ldr; the output is zeroed first and
// every tile adds its product in tile order.
rsvd_status apass_streamed(StreamState* s, const rsvd_matrix& Ah, int trans, int prec, int r, const void* X,
                           void* Y, int64_t ldr, int* status, cudaStream_t st) {
  const int64_t m = Ah.m, n = Ah.n;
  const size_t esz = Ah.dtype == RSVD_F64 ? 8 : 4;
  const int64_t M = trans ? n : m;
  const int64_t Tm = cdiv(m, s->mb), Tn = cdiv(n, s->nb);
  RSVD_CUDA(cudaMemsetAsync(Y, 0, (size_t)M * ldr * esz, st));
  for (int64_t I = 0; I < Tm; ++I) {
    for (int64_t J = 0; J < Tn; ++J) {
      const int64_t t = I * Tn + J;
      const int64_t row0 = I * s->mb, col0 = J * s->nb;
      const int64_t rows = (row0 + s->mb < m ? s->mb : m - row0);
      const int64_t cols = (col0 + s->nb < n ? s->nb : n - col0);
      const char* Xc = static_cast<const char*>(X);
      char* Yc = static_cast<char*>(Y);
      const bool c16 = s->cache16 && t < (int64_t)s->cache.size();
      const float* Xt = reinterpret_cast<const float*>(Xc + (size_t)(trans ? row0 : col0) * ldr * esz);
      float* Yt = reinterpret_cast<float*>(Yc + (size_t)(trans ? col0 : row0) * ldr * esz);
      if (c16 && s->cache_valid[t] && prec == RSVD_PREC_BF16) {  // the resident BF16 copy
        Bf16Source b;
        b.data = static_cast<const uint16_t*>(s->cache[t]);
        b.m = rows;
        b.n = cols;
        b.ld = s->ld16;
        RSVD_TRY(tc_apass_from_16(b, trans, prec, r, Xt, ldr, Yt, ldr, s->ws, s->ws_bytes, status, st, true));
        continue;
      }
      rsvd_matrix T;
      bool cached;
      RSVD_TRY(fetch_tile(s, Ah, t, row0, col0, rows, cols, esz, st, &T, &cached));
      if (c16 && !trans && prec == RSVD_PREC_BF16 && !s->cache_valid[t]) {
        // the first BF16 forward pass over the tile this run: multiply it and
        // keep its BF16 copy
        RSVD_TRY(tc_apass_from_f32(T, 0, prec, r, Xt, ldr, Yt, ldr, 0, 0, s->ws, s->ws_bytes, status, st, true,
                                   static_cast<uint16_t*>(s->cache[t]), s->ld16));
        s->cache_valid[t] = 1;
      } else if (!trans)
        RSVD_TRY(apass_dense(T, 0, prec, r, Xc + (size_t)col0 * ldr * esz, ldr, Yc + (size_t)row0 * ldr * esz, ldr,
                             0, 0, s->ws, s->ws_bytes, status, st, true));
      else
        RSVD_TRY(apass_dense(T, 1, prec, r, Xc + (size_t)row0 * ldr * esz, ldr, Yc + (size_t)col0 * ldr * esz, ldr,
                             0, 0, s->ws, s->ws_bytes, status, st, true));
      if (!cached) RSVD_CUDA(cudaEventRecord(s->freed[slot_of(s, t)], st));
    }
  }
  return RSVD_OK;
}

// One fused power sweep over full-width row panels (Section 2.2, Eq. (3) with
// the product A^T (A W) grouped per panel): for each row panel A_I, in order,
// Y_I = A_I W and then Z += A_I^T Y_I with the panel still on the device, so A
// crosses the host link once per sweep instead of twice.  W and Z: n x r
// (leading dimension ldr); Z is zeroed first.  prec_t is the precision of the
// products A_I^T Y_I (BF16 plans carry Y_I as two BF16 parts there).
rsvd_status sweep_streamed(StreamState* s, const rsvd_matrix& Ah, int prec, int prec_t, int r, const void* W,
                           void* Z, int64_t ldr, int* status, cudaStream_t st) {
  const int64_t m = Ah.m, n = Ah.n;
  if (s->nb < n) return fail(RSVD_ERR_UNSUPPORTED, "rsvd_run: fused sweeps stream full-width row panels (nb = n)");
  const size_t esz = Ah.dtype == RSVD_F64 ? 8 : 4;
  const int64_t Tm = cdiv(m, s->mb);
  RSVD_CUDA(cudaMemsetAsync(Z, 0, (size_t)n * ldr * esz, st));
  for (int64_t I = 0; I < Tm; ++I) {
    const int64_t row0 = I * s->mb;
    const int64_t rows = (row0 + s->mb < m ? s->mb : m - row0);
    rsvd_matrix T;
    bool cached;
    RSVD_TRY(fetch_tile(s, Ah, I, row0, 0, rows, n, esz, st, &T, &cached));
    RSVD_TRY(apass_dense(T, 0, prec, r, W, ldr, s->ytile, ldr, 0, 0, s->ws, s->ws_bytes, status, st, false));
    RSVD_TRY(apass_dense(T, 1, prec_t, r, s->ytile, ldr, Z, ldr, 0, 0, s->ws, s->ws_bytes, status, st, true));
    if (!cached) RSVD_CUDA(cudaEventRecord(s->freed[slot_of(s, I)], st));
  }
  return RSVD_OK;
}

}  // namespace rsvd
