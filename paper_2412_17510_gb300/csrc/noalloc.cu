// noalloc.cu -- multiple-precision CSR SpMV that allocates no memory.
//
// For callers that cannot allocate device memory at the time they multiply:
// a process whose device memory has been handed in full to its own pool or
// arena at start-up (so a cudaMalloc would fail or break its accounting),
// or a latency-critical loop that cannot afford cudaMalloc / cudaFree, which
// synchronise the device.  Such a caller keeps the matrix in its own device
// buffers as plain CSR arrays and calls mpspmv_spmv_csr_noalloc; no handle is
// created.
//
// The only scratch the product needs -- the partial sums of rows that cross
// a run boundary -- lives in the file-scope array below, fixed at load time.
// Every GPU that loads the library holds it (32 MiB) until the process exits.
#include <mutex>

#include "internal.h"
#include "mp_arith.cuh"

using namespace mpk;

namespace {

constexpr int kRun = 16;         // stored entries summed by one thread
constexpr int kThreadsNA = 128;
constexpr int64_t kScratchDoubles = int64_t(1) << 22;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).  The address
// belongs to the device's primary context and is cached for the life of the
// process: after cudaDeviceReset this entry point must not be called again.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    mps_note_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    return MPSPMV_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return MPSPMV_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      mps_note_cuda_error(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
      return MPSPMV_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MPSPMV_OK;
}

// first row whose entries reach past position k (the row holding entry k)
__device__ __forceinline__ int64_t row_of(const int64_t* __restrict__ indptr, int64_t nrows, int64_t k) {
  int64_t lo = 0, hi = nrows - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(indptr + mid + 1) > k) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <int L, bool CPLX>
__device__ __forceinline__ void put(double* __restrict__ y, int64_t n, int64_t r, const mp<L>& a, const mp<L>& b) {
#pragma unroll
  for (int l = 0; l < L; l++) y[(int64_t)l * n + r] = a.v[l];
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) y[(int64_t)(L + l) * n + r] = b.v[l];
  }
}

template <int L, bool CPLX>
__device__ __forceinline__ void put_carry(double* __restrict__ carry, int64_t nchunks, int w, int64_t c,
                                          const mp<L>& a, const mp<L>& b) {
  constexpr int P = CPLX ? 2 * L : L;
#pragma unroll
  for (int p = 0; p < P; p++) carry[(int64_t)(w * P + p) * nchunks + c] = p < L ? a.v[p % L] : b.v[p % L];
}

// One thread per run of kRun entries, summed left to right (one MP multiply
// and one MP add per entry; complex in the order of Eq. complex_spmv).
template <int L, bool CPLX>
__global__ void __launch_bounds__(kThreadsNA) noalloc_runs(int64_t nrows, int64_t nnz, int64_t nchunks,
                                                           const int64_t* __restrict__ indptr,
                                                           const int32_t* __restrict__ indices,
                                                           const double* __restrict__ vals,
                                                           const double* __restrict__ x, int64_t ncols,
                                                           double* __restrict__ y, double* __restrict__ carry) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  const int64_t k0 = c * kRun, k1 = min(k0 + (int64_t)kRun, nnz);
  int64_t row = row_of(indptr, nrows, k0);
  const int64_t first_row = row;
  const bool first_partial = __ldg(indptr + row) < k0;
  int64_t rend = __ldg(indptr + row + 1);
  const mp<L> z = mp_zero<L>();
  if (c == 0)
    for (int64_t r = 0; r < row; r++) put<L, CPLX>(y, nrows, r, z, z);
  mp<L> sr = z, si = z;
  bool have = false;
  for (int64_t k = k0; k < k1; k++) {
    const int64_t j = __ldg(indices + k);
    mp<L> a, xr;
#pragma unroll
    for (int l = 0; l < L; l++) {
      a.v[l] = __ldg(vals + (int64_t)l * nnz + k);
      xr.v[l] = __ldg(x + (int64_t)l * ncols + j);
    }
    sr = mp_add<L>(sr, mp_mul<L>(a, xr));
    if (CPLX) {
      mp<L> ai, xi;
#pragma unroll
      for (int l = 0; l < L; l++) {
        ai.v[l] = __ldg(vals + (int64_t)(L + l) * nnz + k);
        xi.v[l] = __ldg(x + (int64_t)(L + l) * ncols + j);
      }
      sr = mp_add<L>(sr, mp_neg<L>(mp_mul<L>(ai, xi)));
      si = mp_add<L>(si, mp_mul<L>(a, xi));
      si = mp_add<L>(si, mp_mul<L>(ai, xr));
    }
    have = true;
    if (k + 1 == rend) {
      if (row == first_row && first_partial) put_carry<L, CPLX>(carry, nchunks, 0, c, sr, si);
      else put<L, CPLX>(y, nrows, row, sr, si);
      sr = z;
      si = z;
      have = false;
      row++;
      while (row < nrows && __ldg(indptr + row + 1) == k + 1) put<L, CPLX>(y, nrows, row++, z, z);
      rend = row < nrows ? __ldg(indptr + row + 1) : INT64_MAX;
    }
  }
  if (have) put_carry<L, CPLX>(carry, nchunks, (row == first_row && first_partial) ? 0 : 1, c, sr, si);
}

// Rows that cross a run boundary: partial of the starting run, then the
// partials of the following runs in order.
template <int L, bool CPLX>
__global__ void __launch_bounds__(kThreadsNA) noalloc_combine(int64_t nrows, int64_t nchunks,
                                                              const int64_t* __restrict__ indptr,
                                                              double* __restrict__ y,
                                                              const double* __restrict__ carry) {
  constexpr int P = CPLX ? 2 * L : L;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int64_t b = __ldg(indptr + r), e = __ldg(indptr + r + 1);
  if (e <= b) return;
  const int64_t c0 = b / kRun, c1 = (e - 1) / kRun;
  if (c0 == c1) return;
  mp<L> sr, si;
#pragma unroll
  for (int l = 0; l < L; l++) {
    sr.v[l] = carry[(int64_t)(P + l) * nchunks + c0];
    si.v[l] = CPLX ? carry[(int64_t)(P + L + l) * nchunks + c0] : 0.0;
  }
  for (int64_t c = c0 + 1; c <= c1; c++) {
    mp<L> ar, ai;
#pragma unroll
    for (int l = 0; l < L; l++) ar.v[l] = carry[(int64_t)l * nchunks + c];
    sr = mp_add<L>(sr, ar);
    if (CPLX) {
#pragma unroll
      for (int l = 0; l < L; l++) ai.v[l] = carry[(int64_t)(L + l) * nchunks + c];
      si = mp_add<L>(si, ai);
    }
  }
  put<L, CPLX>(y, nrows, r, sr, si);
}

__global__ void noalloc_zero(double* y, int64_t count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count) y[t] = 0.0;
}

template <int L, bool CPLX>
int run(int64_t nrows, int64_t ncols, const int64_t* indptr, const int32_t* indices, const double* vals, int64_t nnz,
        const double* x, double* y, double* carry, cudaStream_t s) {
  constexpr int P = CPLX ? 2 * L : L;
  if (nnz == 0) {
    const int64_t cnt = (int64_t)P * nrows;
    if (cnt > 0) noalloc_zero<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(y, cnt);
    MPS_CUDA(cudaGetLastError());
    return MPSPMV_OK;
  }
  const int64_t nchunks = (nnz + kRun - 1) / kRun;
  noalloc_runs<L, CPLX><<<(unsigned)((nchunks + kThreadsNA - 1) / kThreadsNA), kThreadsNA, 0, s>>>(
      nrows, nnz, nchunks, indptr, indices, vals, x, ncols, y, carry);
  MPS_CUDA(cudaGetLastError());
  noalloc_combine<L, CPLX><<<(unsigned)((nrows + kThreadsNA - 1) / kThreadsNA), kThreadsNA, 0, s>>>(
      nrows, nchunks, indptr, y, carry);
  MPS_CUDA(cudaGetLastError());
  return MPSPMV_OK;
}

// Largest entry count the scratch array holds: two partial sums of P
// components per run of kRun entries.
int64_t max_nnz(int prec, bool cplx) {
  const int64_t P = cplx ? 2 * prec : prec;
  return kScratchDoubles / (2 * P) * kRun;
}

}  // namespace

extern "C" int mpspmv_spmv_csr_noalloc(int prec, unsigned flags, int64_t nrows, int64_t ncols, int64_t nnz,
                                       const int64_t* indptr, const int32_t* indices, const double* vals,
                                       const double* x, double* y, void* stream) {
  if (prec < 1 || prec > 4 || (flags & ~MPSPMV_COMPLEX) || nrows < 0 || ncols < 0 || nnz < 0) return MPSPMV_EINVAL;
  const bool cplx = flags & MPSPMV_COMPLEX;
  if (nnz > max_nnz(prec, cplx)) return MPSPMV_EINVAL;
  // The set-up (loading this file's module, which places the scratch array
  // on the device, and looking up its address) runs on the first call on a
  // device, also for nrows == 0: such a call does only the set-up.
  double* carry = nullptr;
  int st = scratch_address(&carry);
  if (st != MPSPMV_OK) return st;
  if (nrows == 0) return MPSPMV_OK;
  if (!indptr || !y || (nnz > 0 && (!indices || !vals || !x))) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  switch (prec * 2 + (cplx ? 1 : 0)) {
    case 2: return run<1, false>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 3: return run<1, true>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 4: return run<2, false>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 5: return run<2, true>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 6: return run<3, false>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 7: return run<3, true>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 8: return run<4, false>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
    case 9: return run<4, true>(nrows, ncols, indptr, indices, vals, nnz, x, y, carry, s);
  }
  return MPSPMV_EINVAL;
}
