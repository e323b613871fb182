// internal.h -- handle layout and launch helpers shared by the library's
// translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mpspmv.h"

#define MPS_CUDA(call)                              \
  do {                                              \
    cudaError_t _e = (call);                        \
    if (_e != cudaSuccess) {                        \
      mps_note_cuda_error(_e, #call, __FILE__, __LINE__); \
      return MPSPMV_ECUDA;                          \
    }                                               \
  } while (0)

void mps_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Device view of a matrix, passed to kernels by value.
//
// Stored entries are cut into runs ("chunks") of K consecutive entries in
// CSR order; chunk c is summed by one thread.  Runs are grouped 32 at a time
// into tiles whose entries are stored transposed (entry j of the chunk in
// lane l of tile t sits at t*32*K + j*32 + l), so the 32 threads of a warp
// read 32 consecutive values per step.  Every value plane and the column
// array use this tiled order; tlen is the padded length of one plane.
struct DevMat {
  int64_t nrows, ncols, nnz, nchunks, tlen;
  int32_t K;
  const int64_t* indptr;    // nrows + 1, CSR row starts (in entry order)
  const int32_t* cols;      // tlen, tiled
  const double* vals;       // Pv planes of tlen, tiled
  const int64_t* chunk_row; // nchunks: the row holding entry c*K
  const int64_t* split_rows;// rows whose entries span > 1 chunk: the nshort rows
                            // spanning at most kLongSpan chunks, then the rest
  int64_t nsplit, nshort;
};

// Rows whose entries span more than this many chunks are combined by a warp.
constexpr int kLongSpan = 32;

// Words per row of the finished-row buffer of real wide-x products over runs:
// the row accumulator's digit differences (at most 11 digits, QD) and one
// word with its window base (low half) and flush flags (high half); 96
// bytes, three DRAM sectors.
constexpr int kRowDigWords = 12;

struct mpspmv_mat {
  int device;
  int L, P, Pv;  // components, vector planes, stored value planes
  bool cplx, mixed;
  bool exact = false;  // MPSPMV_EXACT_ACC: products on the binary64 pipe, exact integer accumulation
  bool dstore = false; // exact arithmetic on binary64 data: only the leading components are stored and
                       // the products take the MP x binary64 forms (the dropped products are exactly 0)
  unsigned flags;
  int64_t nrows, ncols, nnz, max_row_nnz;
  int32_t K;
  int64_t nchunks, ntiles, tlen, nsplit, nshort;
  int64_t* d_indptr = nullptr;
  int32_t* d_cols = nullptr;
  double* d_vals = nullptr;
  int64_t* d_chunk_row = nullptr;
  int64_t* d_split = nullptr;
  double* d_carry = nullptr;      // 2 * P * nchunks * carry_k
  int carry_k = 0;                // right-hand sides the carry buffer holds
  double* d_xint = nullptr;       // exact handles: x with the P components of a column adjacent
  uint32_t* d_xwide = nullptr;    // exact handles with one value plane: the wide-x records of x (wide.cuh)
  int64_t* d_rowdig = nullptr;    // real wide-x products over runs: per row, the finished row's digits
                                  // (kRowDigWords words) for the finishing pass
  // Exact handles with short, evenly sized rows: a sliced-ELL copy for
  // single-vector products (slices of 32 rows, entry q of row r at
  // slice_ptr[r / 32] + 32 q + r % 32), one thread per row.
  int64_t sell_len = 0;           // slots per value plane (0: no copy)
  int64_t* d_slice_ptr = nullptr; // nrows / 32 + 1 slice offsets
  int32_t* d_sell_cols = nullptr;
  double* d_sell_vals = nullptr;  // Pv planes of sell_len
  double* d_xbuf = nullptr;       // host-buffer entry points
  double* d_ybuf = nullptr;
  double* d_kws = nullptr;        // Krylov vectors and reduction partials
  int64_t kws_len = 0;
  struct KrylovState* d_kstate = nullptr;
  int64_t device_bytes = 0;
  std::vector<int64_t> h_indptr;  // host copy of the row offsets (re-planning)
  mpspmv_mat* tr = nullptr;       // A^T, built from the swapped triplets (MPSPMV_TRANSPOSE)

  DevMat view() const {
    DevMat m;
    m.nrows = nrows; m.ncols = ncols; m.nnz = nnz; m.nchunks = nchunks; m.tlen = tlen; m.K = K;
    m.indptr = d_indptr; m.cols = d_cols; m.vals = d_vals; m.chunk_row = d_chunk_row;
    m.split_rows = d_split; m.nsplit = nsplit; m.nshort = nshort;
    return m;
  }
};

// Launchers implemented in spmv.cu
int mps_build_tiles(mpspmv_mat* h, const double* d_sorted_vals, int64_t nin, int vin_limbs,
                    const int64_t* d_run_start, const int64_t* d_unique_cols_src, cudaStream_t s);
// Sliced-ELL copy of a built matrix (exact handles with short, evenly sized
// rows); no-op when the rows do not qualify.
int mps_build_sell(mpspmv_mat* h, cudaStream_t s);
int mps_launch_spmv(const mpspmv_mat* h, const double* x, double* y, cudaStream_t s);
// SpMV whose kernels do nothing unless *gate == 0 (device flag, e.g. the
// status word of a Krylov solver replayed from a CUDA graph).
int mps_launch_spmv_if_running(const mpspmv_mat* h, const double* x, double* y, const void* gate,
                               cudaStream_t s);
int mps_launch_spmm(mpspmv_mat* h, int k, const double* X, int64_t ldx, double* Y, int64_t ldy,
                    cudaStream_t s);
int mps_ensure_carry(mpspmv_mat* h, int k);
// Run plan for runs of K entries: chunk_row[c] = row holding entry c*K; split
// = rows spanning more than one run, the nshort spanning at most kLongSpan
// runs first.
void mps_plan(const int64_t* indptr, int64_t nrows, int64_t nnz, int32_t K, std::vector<int64_t>& chunk_row,
              std::vector<int64_t>& split, int64_t& nshort);
// Re-cut the stored entries of h into runs of K entries (tiles, plan, carry).
int mps_retile(mpspmv_mat* h, int32_t K, cudaStream_t s);

static inline cudaStream_t mps_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
