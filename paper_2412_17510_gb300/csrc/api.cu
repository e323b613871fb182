// api.cu -- C ABI: matrix creation from COO / Matrix Market triplets, SpMV,
// SpMM, handle queries (arXiv 2412.17510, Section 3).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace {
thread_local char g_last_cuda[256] = {0};

template <typename T>
int dev_alloc(mpspmv_mat* h, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return MPSPMV_ENOMEM;
    mps_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
    return MPSPMV_ECUDA;
  }
  h->device_bytes += (int64_t)(sizeof(T) * (size_t)count);
  return MPSPMV_OK;
}

void free_handle(mpspmv_mat* h) {
  if (!h) return;
  free_handle(h->tr);
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaFree(h->d_indptr);
  cudaFree(h->d_cols);
  cudaFree(h->d_vals);
  cudaFree(h->d_chunk_row);
  cudaFree(h->d_split);
  cudaFree(h->d_carry);
  cudaFree(h->d_xint);
  cudaFree(h->d_xwide);
  cudaFree(h->d_rowdig);
  cudaFree(h->d_slice_ptr);
  cudaFree(h->d_sell_cols);
  cudaFree(h->d_sell_vals);
  cudaFree(h->d_xbuf);
  cudaFree(h->d_ybuf);
  cudaFree(h->d_kws);
  cudaFree(h->d_kstate);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  delete h;
}

// Entries per run: the longest of kmax, kmax/2, ..., 4 that still leaves
// about four waves of threads on 152 SMs (768 resident threads each).  Long
// runs mean fewer rows cut by run boundaries, hence fewer partial sums to
// combine.  kmax is 128 for exact accumulation (each cut row costs two
// flushes and a digit combine; on the power-law matrix n = 1e6 runs of 128
// instead of 64 took the QD product from 5.23 to 5.06 ms) and 64 for the
// paper-order sums.
int32_t pick_chunk(int64_t nnz, int32_t kmax) {
  int32_t K = kmax;
  while (K > 4 && nnz / K < (int64_t)152 * 768 * 4) K >>= 1;
  return K;
}

}  // namespace

void mps_plan(const int64_t* indptr, int64_t nrows, int64_t nnz, int32_t K, std::vector<int64_t>& chunk_row,
              std::vector<int64_t>& split, int64_t& nshort) {
  const int64_t nchunks = (nnz + K - 1) / K;
  chunk_row.assign(nchunks, 0);
  int64_t r = 0;
  for (int64_t c = 0; c < nchunks; c++) {
    const int64_t k0 = c * K;
    while (indptr[r + 1] <= k0) r++;
    chunk_row[c] = r;
  }
  // rows cut by run boundaries: short spans first, then the long ones
  split.clear();
  std::vector<int64_t> split_long;
  for (int64_t i = 0; i < nrows; i++) {
    if (indptr[i + 1] <= indptr[i]) continue;
    const int64_t span = (indptr[i + 1] - 1) / K - indptr[i] / K;
    if (span == 0) continue;
    (span <= kLongSpan ? split : split_long).push_back(i);
  }
  nshort = (int64_t)split.size();
  split.insert(split.end(), split_long.begin(), split_long.end());
}

namespace {

struct DeviceScratch {
  std::vector<void*> ptrs;
  ~DeviceScratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  int alloc(T** p, int64_t count) {
    if (count <= 0) count = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)count) != cudaSuccess) {
      cudaGetLastError();
      return MPSPMV_ENOMEM;
    }
    ptrs.push_back(*p);
    return MPSPMV_OK;
  }
};

int create_impl(mpspmv_h* out, int64_t nrows, int64_t ncols, int64_t nnz_in, const int64_t* row,
                const int64_t* col, const double* val, int val_limbs, int prec, unsigned flags,
                cudaStream_t s) {
  if (!out) return MPSPMV_EINVAL;
  *out = nullptr;
  if (nrows < 0 || ncols < 0 || nnz_in < 0 || nrows >= INT32_MAX || ncols >= INT32_MAX) return MPSPMV_EINVAL;
  if (prec < 1 || prec > 4) return MPSPMV_EINVAL;
  if (flags & ~(MPSPMV_COMPLEX | MPSPMV_MIXED | MPSPMV_SYMMETRIC | MPSPMV_ONE_BASED | MPSPMV_EXACT_ACC |
                MPSPMV_TRANSPOSE))
    return MPSPMV_EINVAL;
  const bool cplx = flags & MPSPMV_COMPLEX, mixed = flags & MPSPMV_MIXED;
  if (mixed && (val_limbs != 1 || prec == 1)) return MPSPMV_EINVAL;
  if (val_limbs < 1 || val_limbs > prec) return MPSPMV_EINVAL;
  if (nnz_in > 0 && (!row || !col || !val)) return MPSPMV_EINVAL;
  if ((flags & MPSPMV_SYMMETRIC) && nrows != ncols) return MPSPMV_EINVAL;
  const int V = cplx ? 2 : 1;
  const int vplanes = V * val_limbs;
  const int64_t base = (flags & MPSPMV_ONE_BASED) ? 1 : 0;

  // -- validate and (optionally) expand the symmetric triangle -------------
  int64_t nsym = 0;
  for (int64_t k = 0; k < nnz_in; k++) {
    const int64_t r = row[k] - base, c = col[k] - base;
    if (r < 0 || r >= nrows || c < 0 || c >= ncols) return MPSPMV_EINVAL;
    if ((flags & MPSPMV_SYMMETRIC) && r != c) nsym++;
  }
  for (int64_t q = 0; q < (int64_t)vplanes * nnz_in; q++)
    if (!std::isfinite(val[q])) return MPSPMV_EINVAL;
  const int64_t nin = nnz_in + nsym;
  std::vector<int64_t> R, C;
  const int64_t* pr = row;
  const int64_t* pc = col;
  std::vector<double> VX;
  const double* pv = val;
  if (base || nsym) {
    R.resize(nin);
    C.resize(nin);
    for (int64_t k = 0; k < nnz_in; k++) {
      R[k] = row[k] - base;
      C[k] = col[k] - base;
    }
    int64_t t = nnz_in;
    std::vector<int64_t> src;
    if (nsym) {
      src.reserve(nsym);
      for (int64_t k = 0; k < nnz_in; k++)
        if (R[k] != C[k]) {
          R[t] = C[k];
          C[t] = R[k];
          src.push_back(k);
          t++;
        }
      VX.resize((size_t)vplanes * nin);
      for (int q = 0; q < vplanes; q++) {
        std::memcpy(&VX[(size_t)q * nin], val + (size_t)q * nnz_in, sizeof(double) * nnz_in);
        for (int64_t e = 0; e < nsym; e++) VX[(size_t)q * nin + nnz_in + e] = val[(size_t)q * nnz_in + src[e]];
      }
      pv = VX.data();
    }
    pr = R.data();
    pc = C.data();
  }

  // -- order by (row, col), stable; find duplicate runs ----------------------
  bool sorted = true;
  for (int64_t k = 1; k < nin && sorted; k++)
    if (pr[k] < pr[k - 1] || (pr[k] == pr[k - 1] && pc[k] < pc[k - 1])) sorted = false;
  std::vector<int64_t> perm;
  if (!sorted) {
    perm.resize(nin);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) {
      return pr[a] != pr[b] ? pr[a] < pr[b] : pc[a] < pc[b];
    });
  }
  auto at = [&](int64_t t) { return sorted ? t : perm[t]; };
  std::vector<int64_t> run_start;
  bool dups = false;
  for (int64_t t = 1; t < nin; t++)
    if (pr[at(t)] == pr[at(t - 1)] && pc[at(t)] == pc[at(t - 1)]) {
      dups = true;
      break;
    }
  int64_t nnz = nin;
  if (dups) {
    run_start.reserve(nin + 1);
    for (int64_t t = 0; t < nin; t++)
      if (t == 0 || pr[at(t)] != pr[at(t - 1)] || pc[at(t)] != pc[at(t - 1)]) run_start.push_back(t);
    nnz = (int64_t)run_start.size();
    run_start.push_back(nin);
  }
  auto ustart = [&](int64_t u) { return dups ? run_start[u] : u; };

  // -- CSR row pointers and the run plan (host) ------------------------------
  std::vector<int64_t> indptr(nrows + 1, 0);
  int64_t maxrow = 0;
  for (int64_t u = 0; u < nnz; u++) indptr[pr[at(ustart(u))] + 1]++;
  for (int64_t i = 0; i < nrows; i++) {
    maxrow = std::max(maxrow, indptr[i + 1]);
    indptr[i + 1] += indptr[i];
  }
  const int32_t K = pick_chunk(nnz, (flags & MPSPMV_EXACT_ACC) ? 128 : 64);
  const int64_t nchunks = (nnz + K - 1) / K;
  const int64_t ntiles = (nchunks + 31) / 32;
  const int64_t tlen = ntiles * 32 * (int64_t)K;
  std::vector<int64_t> chunk_row, split;
  int64_t nshort = 0;
  mps_plan(indptr.data(), nrows, nnz, K, chunk_row, split, nshort);

  // -- handle and device arrays ---------------------------------------------
  mpspmv_mat* h = new mpspmv_mat();
  cudaGetDevice(&h->device);
  h->L = prec;
  h->cplx = cplx;
  h->mixed = mixed;
  h->exact = (flags & MPSPMV_EXACT_ACC) != 0;
  // Exact accumulation of binary64 data (one value component, no duplicates
  // to sum): every product of a zero lower component is exactly zero, so
  // storing the leading components only and using the MP x binary64 product
  // forms gives the same bits with less work and fewer bytes.
  h->dstore = h->exact && !mixed && val_limbs == 1 && !dups && prec > 1;
  h->flags = flags;
  h->P = cplx ? 2 * prec : prec;
  h->Pv = (mixed || h->dstore) ? V : h->P;
  h->nrows = nrows;
  h->ncols = ncols;
  h->nnz = nnz;
  h->max_row_nnz = maxrow;
  h->K = K;
  h->nchunks = nchunks;
  h->ntiles = ntiles;
  h->tlen = tlen;
  h->nsplit = (int64_t)split.size();
  h->nshort = nshort;
  h->h_indptr = indptr;
  int st = MPSPMV_OK;
#define TRY(x)                     \
  do {                             \
    st = (x);                      \
    if (st != MPSPMV_OK) goto fail; \
  } while (0)
  {
    TRY(dev_alloc(h, &h->d_indptr, nrows + 1));
    TRY(dev_alloc(h, &h->d_cols, tlen));
    TRY(dev_alloc(h, &h->d_vals, (int64_t)h->Pv * tlen));
    TRY(dev_alloc(h, &h->d_chunk_row, nchunks));
    TRY(dev_alloc(h, &h->d_split, h->nsplit));
    if (h->exact && prec > 1 && h->Pv == V) {
      // one value plane: single-vector products take the wide-x form, whose
      // records (8 words per column part) replace the interleaved copy
      double* xw = nullptr;
      TRY(dev_alloc(h, &xw, (int64_t)V * 4 * ncols));
      h->d_xwide = reinterpret_cast<uint32_t*>(xw);
    } else if (h->exact && h->P > 1) {
      TRY(dev_alloc(h, &h->d_xint, (int64_t)h->P * ncols));
    }
    TRY(mps_ensure_carry(h, 1));
    if (cudaMemcpyAsync(h->d_indptr, indptr.data(), sizeof(int64_t) * (nrows + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        (nchunks && cudaMemcpyAsync(h->d_chunk_row, chunk_row.data(), sizeof(int64_t) * nchunks,
                                    cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        (h->nsplit && cudaMemcpyAsync(h->d_split, split.data(), sizeof(int64_t) * h->nsplit, cudaMemcpyHostToDevice,
                                      s) != cudaSuccess) ||
        cudaMemsetAsync(h->d_cols, 0, sizeof(int32_t) * tlen, s) != cudaSuccess ||
        cudaMemsetAsync(h->d_vals, 0, sizeof(double) * h->Pv * tlen, s) != cudaSuccess) {
      st = MPSPMV_ECUDA;
      goto fail;
    }
    if (nnz > 0) {
      // sorted triplet values / columns and duplicate runs on the device
      DeviceScratch tmp;
      double* d_vin = nullptr;
      int64_t* d_col = nullptr;
      int64_t* d_runs = nullptr;
      TRY(tmp.alloc(&d_vin, (int64_t)vplanes * nin));
      TRY(tmp.alloc(&d_col, nin));
      std::vector<double> vs;
      std::vector<int64_t> cs;
      const double* vsrc = pv;
      const int64_t* csrc = pc;
      if (!sorted) {
        vs.resize((size_t)vplanes * nin);
        cs.resize(nin);
        for (int q = 0; q < vplanes; q++)
          for (int64_t t = 0; t < nin; t++) vs[(size_t)q * nin + t] = pv[(size_t)q * nin + perm[t]];
        for (int64_t t = 0; t < nin; t++) cs[t] = pc[perm[t]];
        vsrc = vs.data();
        csrc = cs.data();
      }
      if (cudaMemcpyAsync(d_vin, vsrc, sizeof(double) * vplanes * nin, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(d_col, csrc, sizeof(int64_t) * nin, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = MPSPMV_ECUDA;
        goto fail;
      }
      if (dups) {
        TRY(tmp.alloc(&d_runs, nnz + 1));
        if (cudaMemcpyAsync(d_runs, run_start.data(), sizeof(int64_t) * (nnz + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
          st = MPSPMV_ECUDA;
          goto fail;
        }
      }
      TRY(mps_build_tiles(h, d_vin, nin, (mixed || h->dstore) ? 1 : val_limbs, d_runs, d_col, s));
      if (h->exact) TRY(mps_build_sell(h, s));
      if (h->d_xwide && !h->cplx && h->sell_len == 0 && nrows > 0)
        TRY(dev_alloc(h, &h->d_rowdig, nrows * (int64_t)kRowDigWords));
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        st = MPSPMV_ECUDA;
        goto fail;
      }
    } else if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = MPSPMV_ECUDA;
      goto fail;
    }
  }
  // A^T: the same triplets with rows and columns swapped.  Each row of A^T
  // lists its entries in increasing row of A (stable ordering), so a row sum
  // of A^T adds the products in the order of the row-oriented scatter.
  if (flags & MPSPMV_TRANSPOSE) {
    TRY(create_impl(&h->tr, ncols, nrows, nnz_in, col, row, val, val_limbs, prec, flags & ~MPSPMV_TRANSPOSE, s));
    h->device_bytes += h->tr->device_bytes;
  }
#undef TRY
  *out = h;
  return MPSPMV_OK;
fail:
  cudaStreamSynchronize(s);
  free_handle(h);
  return st;
}

}  // namespace

void mps_note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s (%s) at %s:%d", cudaGetErrorString(e), what, file, line);
}

namespace {

// x (host) -> handle buffer, product, handle buffer -> y (host), enqueued on s
int spmv_host_enqueue(mpspmv_h h, const double* x_host, double* y_host, cudaStream_t s) {
  const int64_t xb = sizeof(double) * h->P * std::max<int64_t>(h->ncols, 1);
  const int64_t yb = sizeof(double) * h->P * std::max<int64_t>(h->nrows, 1);
  if (!h->d_xbuf) {
    if (cudaMalloc(&h->d_xbuf, xb) != cudaSuccess) return MPSPMV_ENOMEM;
    h->device_bytes += xb;
  }
  if (!h->d_ybuf) {
    if (cudaMalloc(&h->d_ybuf, yb) != cudaSuccess) return MPSPMV_ENOMEM;
    h->device_bytes += yb;
  }
  MPS_CUDA(cudaMemcpyAsync(h->d_xbuf, x_host, sizeof(double) * h->P * h->ncols, cudaMemcpyHostToDevice, s));
  int st = mps_launch_spmv(h, h->d_xbuf, h->d_ybuf, s);
  if (st != MPSPMV_OK) return st;
  MPS_CUDA(cudaMemcpyAsync(y_host, h->d_ybuf, sizeof(double) * h->P * h->nrows, cudaMemcpyDeviceToHost, s));
  return MPSPMV_OK;
}

}  // namespace

extern "C" {

int mpspmv_create_csr(mpspmv_h* out, int64_t nrows, int64_t ncols, int64_t nnz, const int64_t* row,
                      const int64_t* col, const double* val, int val_limbs, int prec, unsigned flags,
                      void* stream) {
  try {
    return create_impl(out, nrows, ncols, nnz, row, col, val, val_limbs, prec, flags, mps_stream(stream));
  } catch (const std::bad_alloc&) {
    return MPSPMV_ENOMEM;
  } catch (...) {
    return MPSPMV_EINVAL;
  }
}

int mpspmv_destroy(mpspmv_h h) {
  if (!h) return MPSPMV_EINVAL;
  cudaDeviceSynchronize();
  free_handle(h);
  return MPSPMV_OK;
}

const char* mpspmv_strerror(int status) {
  switch (status) {
    case MPSPMV_OK: return "success";
    case MPSPMV_EINVAL: return "invalid argument";
    case MPSPMV_ENOMEM: return "out of memory";
    case MPSPMV_ECUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case MPSPMV_ENOTSUP: return "unsupported combination of options";
    case MPSPMV_EBREAKDOWN: return "Krylov breakdown (zero or non-finite scalar)";
    case MPSPMV_ENOCONV: return "maximum number of iterations reached";
    case MPSPMV_ETIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
  }
}

int mpspmv_get_info(mpspmv_h h, mpspmv_info* info) {
  if (!h || !info) return MPSPMV_EINVAL;
  info->nrows = h->nrows;
  info->ncols = h->ncols;
  info->nnz = h->nnz;
  info->max_row_nnz = h->max_row_nnz;
  info->nchunks = h->nchunks;
  info->nsplit_rows = h->nsplit;
  info->prec = h->L;
  info->planes = h->P;
  info->chunk = h->K;
  info->flags = h->flags;
  info->device_bytes = h->device_bytes;
  info->nlong_rows = h->nsplit - h->nshort;
  info->value_planes = h->Pv;
  info->sell_slots = h->sell_len;
  return MPSPMV_OK;
}

int mpspmv_spmv(mpspmv_h h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return MPSPMV_EINVAL;
  return mps_launch_spmv(h, x, y, mps_stream(stream));
}

int mpspmv_spmtv(mpspmv_h h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return MPSPMV_EINVAL;
  if (!h->tr) return MPSPMV_ENOTSUP;
  return mps_launch_spmv(h->tr, x, y, mps_stream(stream));
}

int mpspmv_spmv_host(mpspmv_h h, const double* x_host, double* y_host, void* stream) {
  if (!h || !x_host || !y_host) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  int st = spmv_host_enqueue(h, x_host, y_host, s);
  if (st != MPSPMV_OK) return st;
  MPS_CUDA(cudaStreamSynchronize(s));
  return MPSPMV_OK;
}

int mpspmv_spmv_host_async(mpspmv_h h, const double* x_host, double* y_host, void* stream) {
  if (!h || !x_host || !y_host) return MPSPMV_EINVAL;
  return spmv_host_enqueue(h, x_host, y_host, mps_stream(stream));
}

int mpspmv_spmm(mpspmv_h h, int k, const double* X, int64_t ldx, double* Y, int64_t ldy, void* stream) {
  if (!h || !X || !Y || k < 1 || k > 32 || ldx < k || ldy < k) return MPSPMV_EINVAL;
  return mps_launch_spmm(h, k, X, ldx, Y, ldy, mps_stream(stream));
}

}  // extern "C"
