// Checkpoint and resume of the precompute's result: a compressed wavelet transfer
// (Section 3, precompute Steps 1-2) written to a file and read back, so that a
// long transfer need not be recomputed.  The paper has no counterpart; this is a
// property of the library.
//
// File layout (little-endian, the byte order of every host this library builds on):
//   char magic[8] = "TSRCMP01";
//   int32 K, J, nu, P, n_rows, n_keep, keep_rule, wavelet;
//   int64 nnz;
//   int64 row_ptr[n_rows + 1]; uint16 col[nnz]; float val[nnz];
//   int32 cidx[nnz]; float cval[nnz]; int64 col_ptr[K J + 1].
// Loading checks the header (magic, ranges, n_rows = 10 P^2 + 2 with P the chart
// side of nu, col_ptr[K J] = row_ptr[n_rows] = nnz) on the host before any device
// work.
#include <cstdio>
#include <cstring>
#include <vector>

#include "handles.cuh"

namespace {

constexpr char kMagic[8] = {'T', 'S', 'R', 'C', 'M', 'P', '0', '1'};

struct Header {
  int32_t K, J, nu, P, n_rows, n_keep, keep_rule, wavelet;
  int64_t nnz;
};

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

template <typename T>
tsr_status to_host(std::vector<T> &h, const T *d, size_t n) {
  h.resize(n);
  if (n) TSR_CUDA(cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost));
  return TSR_OK;
}

template <typename T>
bool write_all(FILE *f, const std::vector<T> &h) {
  return h.empty() || fwrite(h.data(), sizeof(T), h.size(), f) == h.size();
}

template <typename T>
bool read_all(FILE *f, std::vector<T> &h, size_t n) {
  h.resize(n);
  return n == 0 || fread(h.data(), sizeof(T), n, f) == n;
}

template <typename T>
tsr_status upload(T **d, const std::vector<T> &h, size_t n_alloc) {
  TSR_CUDA(cudaMalloc(d, sizeof(T) * (n_alloc ? n_alloc : 1)));
  if (!h.empty()) TSR_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  if (n_alloc > h.size()) TSR_CUDA(cudaMemset(*d + h.size(), 0, sizeof(T) * (n_alloc - h.size())));
  return TSR_OK;
}

}  // namespace

extern "C" tsr_status tsr_compressed_save(const tsr_compressed *c, const char *path) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(c && path, "tsr_compressed_save: NULL argument");
  const size_t KJ = (size_t)c->K * c->J, nnz = (size_t)c->nnz;
  std::vector<int64_t> row_ptr, col_ptr;
  std::vector<uint16_t> col;
  std::vector<float> val, cval;
  std::vector<int32_t> cidx;
  tsr_status st = to_host(row_ptr, c->row_ptr, (size_t)c->n_rows + 1);
  if (st == TSR_OK) st = to_host(col, c->col, nnz);
  if (st == TSR_OK) st = to_host(val, c->val, nnz);
  if (st == TSR_OK) st = to_host(cidx, c->cidx, nnz);
  if (st == TSR_OK) st = to_host(cval, c->cval, nnz);
  if (st == TSR_OK) st = to_host(col_ptr, c->col_ptr, KJ + 1);
  if (st != TSR_OK) return st;
  File out;
  out.f = fopen(path, "wb");
  TSR_CHECK_ARG(out.f, "tsr_compressed_save: cannot open %s for writing", path);
  const Header h{c->K, c->J, c->nu, c->P, c->n_rows, c->n_keep, c->keep_rule, c->wavelet, c->nnz};
  bool ok = fwrite(kMagic, 1, sizeof(kMagic), out.f) == sizeof(kMagic) && fwrite(&h, sizeof(h), 1, out.f) == 1;
  ok = ok && write_all(out.f, row_ptr) && write_all(out.f, col) && write_all(out.f, val) && write_all(out.f, cidx) &&
       write_all(out.f, cval) && write_all(out.f, col_ptr);
  ok = (fflush(out.f) == 0) && ok;
  TSR_CHECK_ARG(ok, "tsr_compressed_save: write to %s failed", path);
  return TSR_OK;
}

extern "C" tsr_status tsr_compressed_load(const char *path, tsr_compressed **out) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(path && out, "tsr_compressed_load: NULL argument");
  *out = nullptr;
  File in;
  in.f = fopen(path, "rb");
  TSR_CHECK_ARG(in.f, "tsr_compressed_load: cannot open %s", path);
  char magic[8];
  Header h;
  TSR_CHECK_ARG(fread(magic, 1, sizeof(magic), in.f) == sizeof(magic) && memcmp(magic, kMagic, sizeof(magic)) == 0,
                "tsr_compressed_load: %s is not a compressed transfer file", path);
  TSR_CHECK_ARG(fread(&h, sizeof(h), 1, in.f) == 1, "tsr_compressed_load: %s: truncated header", path);
  TSR_CHECK_ARG(h.K >= 1 && h.K <= 16 && h.J >= 1 && h.J <= 32 && h.nu >= 1 && h.nu <= 128 &&
                    h.P == tsr::chart_side(h.nu) && h.n_rows == 10 * h.P * h.P + 2 && h.nnz >= 0 &&
                    h.nnz <= (int64_t)h.K * h.J * h.n_rows && (h.keep_rule == 0 || h.keep_rule == 1) &&
                    (h.wavelet == 0 || h.wavelet == 1),
                "tsr_compressed_load: %s: header out of range", path);
  const size_t KJ = (size_t)h.K * h.J, nnz = (size_t)h.nnz;
  std::vector<int64_t> row_ptr, col_ptr;
  std::vector<uint16_t> col;
  std::vector<float> val, cval;
  std::vector<int32_t> cidx;
  const bool ok = read_all(in.f, row_ptr, (size_t)h.n_rows + 1) && read_all(in.f, col, nnz) &&
                  read_all(in.f, val, nnz) && read_all(in.f, cidx, nnz) && read_all(in.f, cval, nnz) &&
                  read_all(in.f, col_ptr, KJ + 1);
  TSR_CHECK_ARG(ok, "tsr_compressed_load: %s: truncated arrays", path);
  TSR_CHECK_ARG(row_ptr[0] == 0 && row_ptr[h.n_rows] == h.nnz && col_ptr[0] == 0 && col_ptr[KJ] == h.nnz,
                "tsr_compressed_load: %s: row or column pointers inconsistent with nnz", path);
  for (size_t q = 0; q < nnz; ++q)
    TSR_CHECK_ARG(col[q] < KJ && cidx[q] >= 0 && cidx[q] < h.n_rows, "tsr_compressed_load: %s: entry %zu out of range",
                  path, q);
  tsr_status st = tsr::require_device();
  if (st != TSR_OK) return st;
  tsr_compressed *c = new tsr_compressed();
  cudaGetDevice(&c->device);
  c->K = h.K;
  c->J = h.J;
  c->nu = h.nu;
  c->P = h.P;
  c->n_rows = h.n_rows;
  c->n_keep = h.n_keep;
  c->keep_rule = h.keep_rule;
  c->wavelet = h.wavelet;
  c->nnz = h.nnz;
  const size_t nnz4 = (nnz + 3) & ~(size_t)3;   // col and val padded to whole groups of 4 entries, as compress does
  st = upload(&c->row_ptr, row_ptr, row_ptr.size());
  if (st == TSR_OK) st = upload(&c->col, col, nnz4);
  if (st == TSR_OK) st = upload(&c->val, val, nnz4);
  if (st == TSR_OK) st = upload(&c->cidx, cidx, nnz);
  if (st == TSR_OK) st = upload(&c->cval, cval, nnz);
  if (st == TSR_OK) st = upload(&c->col_ptr, col_ptr, col_ptr.size());
  if (st != TSR_OK) {
    tsr_compressed_destroy(c);
    return st;
  }
  *out = c;
  return TSR_OK;
}
