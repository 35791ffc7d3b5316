// Persistence and resumption (Section 3.8): after each orthonormalisation of
// the range finder the current basis (Q, m x r, or Z, n x r) is written to a
// checkpoint file together with a header that places it in the execution
// plan (problem shape, seed, precision, the step just completed, a
// fingerprint of A).  A later rsvd_run of a plan with the same parameters on
// the same A reads the header, loads the basis and continues with the next
// step, so an interrupted run redoes only the steps it had not finished.
//
// Steps of the range finder: 0 = Q_0 = orth(A O); 2i+1 = Z_{i+1} =
// orth(A^T Q_i); 2i+2 = Q_{i+1} = orth(A Z_{i+1}); i < q.  The file is written
// to "<path>.tmp" and renamed over <path>, so a crash while writing leaves the
// previous checkpoint intact.
//
// File layout (native byte order): CkptHeader, then the basis panel rows x ldr
// elements of the plan's dtype.  Header and panel carry FNV-1a 64-bit
// checksums; a file whose checksums, magic or version do not match is ignored.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

namespace {

constexpr char kMagic[8] = {'R', 'S', 'V', 'D', 'C', 'K', 'P', '1'};
constexpr uint64_t kFnvOffset = 1469598103934665603ull;
constexpr uint64_t kFnvPrime = 1099511628211ull;

uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = kFnvOffset) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= kFnvPrime;
  }
  return h;
}

uint64_t header_checksum(const CkptHeader& h) {
  CkptHeader c = h;
  c.header_checksum = 0;
  return fnv1a(&c, sizeof(c));
}

// Fingerprint of A: the bit patterns of kSamples entries at fixed, spread
// positions (dense), or of nnz, rowptr samples and entries (CSR), folded with
// FNV-1a on the device side order-independently enough to be deterministic:
// each sample writes its own slot, the host folds the slots in order.
constexpr int kSamples = 1024;

template <typename T>
__global__ void sample_dense_kernel(int64_t m, int64_t n, const T* __restrict__ A, int64_t ld,
                                    unsigned long long* __restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kSamples; t += gridDim.x * blockDim.x) {
    const int64_t i = ((int64_t)t * 7919 + 13) % m, j = ((int64_t)t * 104729 + 7) % n;
    out[t] = (unsigned long long)__double_as_longlong((double)A[i * ld + j]);
  }
}

__global__ void sample_csr_kernel(int64_t m, int64_t nnz, const int32_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ colidx, const float* __restrict__ val,
                                  unsigned long long* __restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kSamples; t += gridDim.x * blockDim.x) {
    const int64_t i = ((int64_t)t * 7919 + 13) % (m + 1);
    unsigned long long v = (unsigned long long)(uint32_t)rowptr[i];
    if (nnz > 0) {
      const int64_t e = ((int64_t)t * 104729 + 7) % nnz;
      v = v * 1099511628211ull ^ ((unsigned long long)(uint32_t)colidx[e] << 32 | __float_as_uint(val[e]));
    }
    out[t] = v;
  }
}

}  // namespace

rsvd_status matrix_fingerprint(const rsvd_matrix& A, uint64_t* out, cudaStream_t st) {
  std::vector<unsigned long long> h(kSamples, 0);
  if (A.location == RSVD_ON_HOST) {
    if (A.kind == RSVD_DENSE) {
      for (int t = 0; t < kSamples; ++t) {
        const int64_t i = ((int64_t)t * 7919 + 13) % A.m, j = ((int64_t)t * 104729 + 7) % A.n;
        double v;
        if (A.dtype == RSVD_F64) v = static_cast<const double*>(A.data)[i * A.ld + j];
        else if (A.dtype == RSVD_BF16 || A.dtype == RSVD_F16)  // the 16-bit pattern itself
          v = (double)static_cast<const uint16_t*>(A.data)[i * A.ld + j];
        else v = (double)static_cast<const float*>(A.data)[i * A.ld + j];
        std::memcpy(&h[t], &v, 8);
      }
    } else {
      // the same samples as sample_csr_kernel, read from the host arrays
      for (int t = 0; t < kSamples; ++t) {
        const int64_t i = ((int64_t)t * 7919 + 13) % (A.m + 1);
        unsigned long long v = (unsigned long long)(uint32_t)A.rowptr[i];
        if (A.nnz > 0) {
          const int64_t e = ((int64_t)t * 104729 + 7) % A.nnz;
          uint32_t vb;
          std::memcpy(&vb, &A.val[e], 4);
          v = v * 1099511628211ull ^ ((unsigned long long)(uint32_t)A.colidx[e] << 32 | vb);
        }
        h[t] = v;
      }
    }
  } else {
    unsigned long long* d = nullptr;
    RSVD_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), kSamples * sizeof(unsigned long long), st));
    if (A.kind == RSVD_DENSE) {
      if (A.dtype == RSVD_F64)
        sample_dense_kernel<double><<<4, 256, 0, st>>>(A.m, A.n, static_cast<const double*>(A.data), A.ld, d);
      else if (A.dtype == RSVD_BF16 || A.dtype == RSVD_F16)
        sample_dense_kernel<uint16_t><<<4, 256, 0, st>>>(A.m, A.n, static_cast<const uint16_t*>(A.data), A.ld, d);
      else
        sample_dense_kernel<float><<<4, 256, 0, st>>>(A.m, A.n, static_cast<const float*>(A.data), A.ld, d);
    } else {
      sample_csr_kernel<<<4, 256, 0, st>>>(A.m, A.nnz, A.rowptr, A.colidx, A.val, d);
    }
    RSVD_CUDA(after_launch());
    RSVD_CUDA(cudaMemcpyAsync(h.data(), d, kSamples * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    RSVD_CUDA(cudaFreeAsync(d, st));
    RSVD_CUDA(cudaStreamSynchronize(st));
  }
  uint64_t f = fnv1a(&A.m, sizeof(A.m));
  f = fnv1a(&A.n, sizeof(A.n), f);
  f = fnv1a(&A.nnz, sizeof(A.nnz), f);
  *out = fnv1a(h.data(), h.size() * sizeof(unsigned long long), f);
  return RSVD_OK;
}

void ckpt_fill_header(CkptHeader* h) {
  std::memcpy(h->magic, kMagic, 8);
  h->version = 1;
  h->header_bytes = sizeof(CkptHeader);
}

rsvd_status ckpt_save(const std::string& path, CkptHeader h, const void* dev_panel, cudaStream_t st) {
  std::vector<char> buf(h.panel_bytes);
  RSVD_CUDA(cudaMemcpyAsync(buf.data(), dev_panel, h.panel_bytes, cudaMemcpyDeviceToHost, st));
  RSVD_CUDA(cudaStreamSynchronize(st));
  ckpt_fill_header(&h);
  h.panel_checksum = fnv1a(buf.data(), buf.size());
  h.header_checksum = header_checksum(h);
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(RSVD_ERR_INVALID_ARG, "checkpoint: cannot open " + tmp + " for writing");
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && (buf.empty() || std::fwrite(buf.data(), buf.size(), 1, f) == 1);
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) {
    std::remove(tmp.c_str());
    return fail(RSVD_ERR_INVALID_ARG, "checkpoint: writing " + tmp + " failed");
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return fail(RSVD_ERR_INVALID_ARG, "checkpoint: cannot rename " + tmp + " to " + path);
  }
  return RSVD_OK;
}

bool ckpt_read_header(const std::string& path, CkptHeader* h) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  const bool ok = std::fread(h, sizeof(*h), 1, f) == 1;
  std::fclose(f);
  if (!ok) return false;
  if (std::memcmp(h->magic, kMagic, 8) != 0 || h->version != 1 || h->header_bytes != sizeof(CkptHeader)) return false;
  return header_checksum(*h) == h->header_checksum;
}

bool ckpt_matches(const CkptHeader& a, const CkptHeader& b) {
  return a.m == b.m && a.n == b.n && a.k == b.k && a.p == b.p && a.q == b.q && a.r == b.r && a.ldr == b.ldr &&
         a.prec == b.prec && a.dtype == b.dtype && a.kind == b.kind && a.seed == b.seed &&
         a.fingerprint == b.fingerprint;
}

int ckpt_try_load(const std::string& path, const CkptHeader& expect, void* dev_q, void* dev_z, cudaStream_t st) {
  CkptHeader h;
  if (!ckpt_read_header(path, &h) || !ckpt_matches(h, expect)) return -1;
  if (h.step < 0 || h.step >= 2 * expect.q + 1) return -1;
  const bool is_q = (h.step % 2) == 0;
  const int64_t rows = is_q ? expect.m : expect.n;
  const size_t esz = expect.dtype == RSVD_F64 ? 8 : 4;
  if (h.panel_rows != rows || h.panel_bytes != (uint64_t)rows * expect.ldr * esz) return -1;
  std::vector<char> buf(h.panel_bytes);
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return -1;
  bool ok = std::fseek(f, (long)sizeof(CkptHeader), SEEK_SET) == 0 &&
            (buf.empty() || std::fread(buf.data(), buf.size(), 1, f) == 1);
  std::fclose(f);
  if (!ok || fnv1a(buf.data(), buf.size()) != h.panel_checksum) return -1;
  if (cudaMemcpyAsync(is_q ? dev_q : dev_z, buf.data(), buf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  return h.step;
}

}  // namespace rsvd

extern "C" rsvd_status rsvd_checkpoint_info(const char* path, rsvd_checkpoint_info_t* out) {
  using namespace rsvd;
  if (!path || !out) return fail(RSVD_ERR_INVALID_ARG, "rsvd_checkpoint_info: NULL argument");
  std::memset(out, 0, sizeof(*out));
  CkptHeader h;
  if (!ckpt_read_header(path, &h)) return fail(RSVD_ERR_INVALID_ARG, "rsvd_checkpoint_info: no valid checkpoint header");
  out->m = h.m; out->n = h.n; out->k = h.k; out->p = h.p; out->q = h.q; out->r = h.r;
  out->prec = h.prec; out->dtype = h.dtype; out->kind = h.kind; out->seed = h.seed;
  out->fingerprint = h.fingerprint; out->step = h.step; out->panel_rows = h.panel_rows;
  out->panel_bytes = h.panel_bytes;
  return RSVD_OK;
}
