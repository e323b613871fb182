// select.cu -- learned precision selector: matrix features on the device and
// a small float32 multilayer perceptron (32 -> 128 -> 128 -> C) trained and
// evaluated by hand-written kernels.  The paper motivates multiple precision
// by the round-off sensitivity of Krylov methods (Section 1, Section 4.2)
// but selects the format by hand; the selector predicts, from cheap matrix
// features, the lowest of binary64 / DD / TD / QD at which CG reaches a target
// residual, and the precision ladder stays as its fallback.
//
// Features (32 floats, feature i below), computed from the stored matrix:
//   0 log10 n              1 log10 nnz            2..5 row length mean, std, min, max
//   6 row length cv        7 row length skewness  8 fraction of empty rows
//   9 bandwidth / n        10..12 diagonal dominance |a_ii| / sum_{j!=i}|a_ij|: min, mean, max
//   13 fraction of diagonally dominant rows
//   14 log10 ||A||_1       15 log10 ||A||_inf     16 log10 ||A||_F
//   17 log10 max|a_ii|     18 log10 min|a_ii|     19 log10 (max|a_ii| / min|a_ii|)
//   20, 21 Gershgorin lower / upper bound divided by ||A||_inf
//   22..29 log10 ||r_k|| / ||b|| of binary64 CG on the system, k = 1..8 (x0 = 0)
//   30 least-squares slope of 22..29 against k
//   31 log10 (||A||_F / max|a_ii|)
// (components other than the leading one of each stored value are ignored;
// log10 of zero is clamped to -300.)
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "krylov.h"
#include "run_body.cuh"

namespace {

constexpr int kFT = 256;

struct RowStats {
  double len, diag, off, rowabs, rowsq, bw;
};

// per row: length, leading component of a_ii, off-diagonal |.| sum, row |.|
// sum, row square sum, max |i - j|; column |.| sums by atomics
__global__ void row_stats_kernel(DevMat m, double* __restrict__ out, double* __restrict__ colsum) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m.nrows) return;
  const int64_t b = m.indptr[r], e = m.indptr[r + 1];
  double diag = 0.0, off = 0.0, sq = 0.0, bw = 0.0;
  for (int64_t u = b; u < e; u++) {
    const int64_t c = u / m.K;
    const int64_t pos = mpk::tile_pos(c, (int)(u - c * m.K), m.K);
    const int64_t j = m.cols[pos];
    const double v = m.vals[pos];
    if (j == r) diag += v;
    else off += fabs(v);
    sq += v * v;
    bw = fmax(bw, fabs((double)(j - r)));
    atomicAdd(colsum + j, fabs(v));
  }
  double* o = out + r * 6;
  o[0] = (double)(e - b);
  o[1] = diag;
  o[2] = off;
  o[3] = off + fabs(diag);
  o[4] = sq;
  o[5] = bw;
}

double lg(double v) { return v > 0.0 ? std::log10(v) : -300.0; }

}  // namespace

// Features of a handle into feat[32] (host).  cg_hist: 8 binary64 CG residual
// ratios supplied by the caller (the ladder computes them with a binary64
// handle); NULL leaves features 22..30 zero.
int mps_features(mpspmv_mat* h, const double* cg_hist, float* feat, cudaStream_t s) {
  const int64_t n = h->nrows;
  std::vector<double> rs((size_t)std::max<int64_t>(n, 1) * 6), cs((size_t)std::max<int64_t>(h->ncols, 1));
  double *d_rs = nullptr, *d_cs = nullptr;
  if (cudaMalloc(&d_rs, sizeof(double) * rs.size()) != cudaSuccess ||
      cudaMalloc(&d_cs, sizeof(double) * cs.size()) != cudaSuccess) {
    cudaFree(d_rs);
    cudaGetLastError();
    return MPSPMV_ENOMEM;
  }
  int st = MPSPMV_OK;
  if (cudaMemsetAsync(d_cs, 0, sizeof(double) * cs.size(), s) != cudaSuccess) st = MPSPMV_ECUDA;
  if (!st && n > 0) {
    row_stats_kernel<<<(unsigned)((n + kFT - 1) / kFT), kFT, 0, s>>>(h->view(), d_rs, d_cs);
    if (cudaGetLastError() != cudaSuccess) st = MPSPMV_ECUDA;
  }
  if (!st && (cudaMemcpyAsync(rs.data(), d_rs, sizeof(double) * rs.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaMemcpyAsync(cs.data(), d_cs, sizeof(double) * cs.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    st = MPSPMV_ECUDA;
  cudaFree(d_rs);
  cudaFree(d_cs);
  if (st) return st;
  // reductions over rows (host, in row order)
  double s1 = 0, s2 = 0, s3 = 0, lmin = 1e300, lmax = 0, empty = 0, bw = 0;
  double dmin = 1e300, dsum = 0, dmax = 0, ndom = 0, ninf = 0, fro = 0, amax = 0, amin = 1e300, glo = 1e300,
         ghi = -1e300;
  for (int64_t r = 0; r < n; r++) {
    const double* o = &rs[(size_t)r * 6];
    const double len = o[0];
    s1 += len;
    s2 += len * len;
    s3 += len * len * len;
    lmin = std::min(lmin, len);
    lmax = std::max(lmax, len);
    if (len == 0) empty += 1;
    bw = std::max(bw, o[5]);
    const double ad = std::fabs(o[1]);
    const double dom = o[2] > 0 ? ad / o[2] : 1e30;
    dmin = std::min(dmin, dom);
    dmax = std::max(dmax, std::min(dom, 1e30));
    dsum += std::min(dom, 1e6);
    if (ad >= o[2]) ndom += 1;
    ninf = std::max(ninf, o[3]);
    fro += o[4];
    amax = std::max(amax, ad);
    amin = std::min(amin, ad);
    glo = std::min(glo, o[1] - o[2]);
    ghi = std::max(ghi, o[1] + o[2]);
  }
  double n1 = 0;
  for (double c : cs) n1 = std::max(n1, c);
  const double nn = std::max<double>((double)n, 1.0);
  const double mean = s1 / nn;
  const double var = std::max(s2 / nn - mean * mean, 0.0);
  const double sd = std::sqrt(var);
  const double m3 = s3 / nn - 3 * mean * s2 / nn + 2 * mean * mean * mean;
  double f[32] = {0};
  f[0] = lg((double)n);
  f[1] = lg((double)h->nnz);
  f[2] = mean;
  f[3] = sd;
  f[4] = n ? lmin : 0;
  f[5] = lmax;
  f[6] = mean > 0 ? sd / mean : 0;
  f[7] = sd > 0 ? m3 / (sd * sd * sd) : 0;
  f[8] = empty / nn;
  f[9] = bw / nn;
  f[10] = lg(dmin);
  f[11] = lg(dsum / nn);
  f[12] = lg(dmax);
  f[13] = ndom / nn;
  f[14] = lg(n1);
  f[15] = lg(ninf);
  f[16] = lg(std::sqrt(fro));
  f[17] = lg(amax);
  f[18] = lg(amin);
  f[19] = f[17] - f[18];
  f[20] = ninf > 0 ? glo / ninf : 0;
  f[21] = ninf > 0 ? ghi / ninf : 0;
  if (cg_hist) {
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int k = 0; k < 8; k++) {
      f[22 + k] = lg(cg_hist[k]);
      sx += k + 1;
      sy += f[22 + k];
      sxx += (k + 1) * (k + 1);
      sxy += (k + 1) * f[22 + k];
    }
    f[30] = (8 * sxy - sx * sy) / (8 * sxx - sx * sx);
  }
  f[31] = lg(std::sqrt(fro)) - lg(amax);
  for (int i = 0; i < 32; i++) feat[i] = (float)f[i];
  return MPSPMV_OK;
}

// ---------------------------------------------------------------------------
// MLP kernels (float32).  Parameters are one device buffer:
//   W1 32x128 | b1 128 | W2 128x128 | b2 128 | W3 128xC | b3 C   (row-major)
// ---------------------------------------------------------------------------
namespace {

constexpr int D0 = 32, D1 = 128, D2 = 128;

struct MlpView {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__host__ __device__ inline int64_t mlp_param_count(int C) {
  return (int64_t)D0 * D1 + D1 + (int64_t)D1 * D2 + D2 + (int64_t)D2 * C + C;
}

__host__ __device__ inline MlpView mlp_view(const float* p, int C) {
  MlpView v;
  v.W1 = p;
  v.b1 = v.W1 + D0 * D1;
  v.W2 = v.b1 + D1;
  v.b2 = v.W2 + D1 * D2;
  v.W3 = v.b2 + D2;
  v.b3 = v.W3 + D2 * C;
  return v;
}

// out[b, j] = act(sum_i in[b, i] W[i, j] + bias[j]); thread per (b, j), the
// sum over i in index order (deterministic).
__global__ void dense_kernel(const float* __restrict__ in, int B, int din, const float* __restrict__ W,
                             const float* __restrict__ bias, int dout, float* __restrict__ z,
                             float* __restrict__ a, int relu) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * dout) return;
  const int b = (int)(t / dout), j = (int)(t - (int64_t)b * dout);
  float acc = bias[j];
  for (int i = 0; i < din; i++) acc = fmaf(in[(int64_t)b * din + i], W[(int64_t)i * dout + j], acc);
  z[t] = acc;
  if (a) a[t] = relu ? fmaxf(acc, 0.0f) : acc;
}

// softmax cross-entropy: d3[b, c] = (p_c - [c == y_b]) / B, loss_b
__global__ void softmax_xent_kernel(const float* __restrict__ z3, const int* __restrict__ y, int B, int C,
                                    float* __restrict__ d3, float* __restrict__ lossb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* z = z3 + (int64_t)b * C;
  float m = z[0];
  for (int c = 1; c < C; c++) m = fmaxf(m, z[c]);
  float s = 0.0f;
  for (int c = 0; c < C; c++) s += expf(z[c] - m);
  const float ls = logf(s);
  for (int c = 0; c < C; c++) {
    const float p = expf(z[c] - m - ls);
    d3[(int64_t)b * C + c] = (p - (c == y[b] ? 1.0f : 0.0f)) / (float)B;
  }
  lossb[b] = -(z[y[b]] - m - ls);
}

// gW[i, j] = sum_b a[b, i] d[b, j]; gb[j] = sum_b d[b, j]   (thread per (i, j))
__global__ void weight_grad_kernel(const float* __restrict__ a, const float* __restrict__ d, int B, int din,
                                   int dout, float* __restrict__ gW, float* __restrict__ gb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)(din + 1) * dout) return;
  const int i = (int)(t / dout), j = (int)(t - (int64_t)i * dout);
  float acc = 0.0f;
  if (i < din) {
    for (int b = 0; b < B; b++) acc = fmaf(a[(int64_t)b * din + i], d[(int64_t)b * dout + j], acc);
    gW[(int64_t)i * dout + j] = acc;
  } else {
    for (int b = 0; b < B; b++) acc += d[(int64_t)b * dout + j];
    gb[j] = acc;
  }
}

// dprev[b, i] = (sum_j d[b, j] W[i, j]) * (zprev[b, i] > 0)
__global__ void back_kernel(const float* __restrict__ d, const float* __restrict__ W, int B, int din, int dout,
                            const float* __restrict__ zprev, float* __restrict__ dprev) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * din) return;
  const int b = (int)(t / din), i = (int)(t - (int64_t)b * din);
  float acc = 0.0f;
  for (int j = 0; j < dout; j++) acc = fmaf(d[(int64_t)b * dout + j], W[(int64_t)i * dout + j], acc);
  dprev[t] = zprev[t] > 0.0f ? acc : 0.0f;
}

__global__ void sgd_kernel(float* __restrict__ p, const float* __restrict__ g, int64_t n, float lr) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) p[t] -= lr * g[t];
}

// Column statistics of n feature vectors (n x D0, row-major): mean and
// population standard deviation of every feature, summed in binary64 in
// sample order (deterministic), rounded to float; a deviation below 1e-6
// becomes 1 (a constant feature passes unscaled).  Xs = (X - mu) / sd with
// the rounded mu and sd, so that the fold below is consistent with it.
// One thread per feature.
__global__ void standardize_kernel(const float* __restrict__ X, int n, float* __restrict__ mu,
                                   float* __restrict__ sd, float* __restrict__ Xs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D0) return;
  double s = 0.0;
  for (int b = 0; b < n; b++) s += (double)X[(int64_t)b * D0 + i];
  const double m = s / n;
  double v = 0.0;
  for (int b = 0; b < n; b++) {
    const double d = (double)X[(int64_t)b * D0 + i] - m;
    v += d * d;
  }
  double sdv = sqrt(v / n);
  if (sdv < 1e-6) sdv = 1.0;
  const float mf = (float)m, sf = (float)sdv;
  mu[i] = mf;
  sd[i] = sf;
  for (int b = 0; b < n; b++) Xs[(int64_t)b * D0 + i] = (float)(((double)X[(int64_t)b * D0 + i] - mf) / sf);
}

// First layer rewritten for raw features: ((x - mu) / sd) W1 + b1 =
// x (W1 / sd[:, None]) + (b1 - (mu / sd) W1).  One thread per hidden unit,
// binary64 arithmetic over the inputs in index order, rounded to float.
__global__ void fold_kernel(float* __restrict__ W1, float* __restrict__ b1, const float* __restrict__ mu,
                            const float* __restrict__ sd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= D1) return;
  double acc = b1[j];
  for (int i = 0; i < D0; i++) acc -= (double)mu[i] / (double)sd[i] * (double)W1[(int64_t)i * D1 + j];
  b1[j] = (float)acc;
  for (int i = 0; i < D0; i++) W1[(int64_t)i * D1 + j] = (float)((double)W1[(int64_t)i * D1 + j] / (double)sd[i]);
}

inline unsigned nb(int64_t n) { return (unsigned)((n + kFT - 1) / kFT); }

struct MlpWork {
  float *z1, *a1, *z2, *a2, *z3, *d3, *d2, *d1, *loss;
};

int mlp_alloc(int B, int C, float** buf, MlpWork& w) {
  const int64_t n = (int64_t)B * (2 * D1 + 2 * D2 + 2 * C + D2 + D1 + 1);
  if (cudaMalloc(buf, sizeof(float) * n) != cudaSuccess) {
    cudaGetLastError();
    return MPSPMV_ENOMEM;
  }
  float* p = *buf;
  w.z1 = p; p += (int64_t)B * D1;
  w.a1 = p; p += (int64_t)B * D1;
  w.z2 = p; p += (int64_t)B * D2;
  w.a2 = p; p += (int64_t)B * D2;
  w.z3 = p; p += (int64_t)B * C;
  w.d3 = p; p += (int64_t)B * C;
  w.d2 = p; p += (int64_t)B * D2;
  w.d1 = p; p += (int64_t)B * D1;
  w.loss = p;
  return MPSPMV_OK;
}

void mlp_forward(const MlpView& v, const float* X, int B, int C, const MlpWork& w, cudaStream_t s) {
  dense_kernel<<<nb((int64_t)B * D1), kFT, 0, s>>>(X, B, D0, v.W1, v.b1, D1, w.z1, w.a1, 1);
  dense_kernel<<<nb((int64_t)B * D2), kFT, 0, s>>>(w.a1, B, D1, v.W2, v.b2, D2, w.z2, w.a2, 1);
  dense_kernel<<<nb((int64_t)B * C), kFT, 0, s>>>(w.a2, B, D2, v.W3, v.b3, C, w.z3, nullptr, 0);
}

// gradients of the mean cross-entropy into g (same layout as the parameters)
void mlp_backward(const MlpView& v, const float* X, const int* y, int B, int C, const MlpWork& w, float* g,
                  cudaStream_t s) {
  MlpView gv = mlp_view(g, C);
  softmax_xent_kernel<<<nb(B), kFT, 0, s>>>(w.z3, y, B, C, w.d3, w.loss);
  weight_grad_kernel<<<nb((int64_t)(D2 + 1) * C), kFT, 0, s>>>(w.a2, w.d3, B, D2, C, const_cast<float*>(gv.W3),
                                                               const_cast<float*>(gv.b3));
  back_kernel<<<nb((int64_t)B * D2), kFT, 0, s>>>(w.d3, v.W3, B, D2, C, w.z2, w.d2);
  weight_grad_kernel<<<nb((int64_t)(D1 + 1) * D2), kFT, 0, s>>>(w.a1, w.d2, B, D1, D2, const_cast<float*>(gv.W2),
                                                                const_cast<float*>(gv.b2));
  back_kernel<<<nb((int64_t)B * D1), kFT, 0, s>>>(w.d2, v.W2, B, D1, D2, w.z1, w.d1);
  weight_grad_kernel<<<nb((int64_t)(D0 + 1) * D1), kFT, 0, s>>>(X, w.d1, B, D0, D1, const_cast<float*>(gv.W1),
                                                                const_cast<float*>(gv.b1));
}

}  // namespace

// class of one feature vector (host floats) = argmax of the logits
int mps_mlp_classify(const float* params, int C, const float* feat, int* cls, cudaStream_t s) {
  float* d = nullptr;
  if (cudaMalloc(&d, sizeof(float) * (D0 + 16)) != cudaSuccess) {
    cudaGetLastError();
    return MPSPMV_ENOMEM;
  }
  float* dl = d + D0;
  float* buf = nullptr;
  MlpWork w;
  int st = mlp_alloc(1, C, &buf, w);
  std::vector<float> lg(C);
  if (!st) {
    cudaMemcpyAsync(d, feat, sizeof(float) * D0, cudaMemcpyHostToDevice, s);
    mlp_forward(mlp_view(params, C), d, 1, C, w, s);
    cudaMemcpyAsync(lg.data(), w.z3, sizeof(float) * C, cudaMemcpyDeviceToHost, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = MPSPMV_ECUDA;
  }
  (void)dl;
  cudaFree(buf);
  cudaFree(d);
  if (st) return st;
  *cls = (int)(std::max_element(lg.begin(), lg.end()) - lg.begin());
  return MPSPMV_OK;
}

extern "C" {

int64_t mpspmv_mlp_param_count(int C) { return C >= 2 && C <= 16 ? mlp_param_count(C) : -1; }

int mpspmv_mlp_forward(const float* params, int C, const float* X, int B, float* logits, void* stream) {
  if (!params || !X || !logits || B < 1 || C < 2 || C > 16) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  float* buf = nullptr;
  MlpWork w;
  int st = mlp_alloc(B, C, &buf, w);
  if (st) return st;
  mlp_forward(mlp_view(params, C), X, B, C, w, s);
  cudaMemcpyAsync(logits, w.z3, sizeof(float) * B * C, cudaMemcpyDeviceToDevice, s);
  st = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess ? MPSPMV_OK : MPSPMV_ECUDA;
  cudaFree(buf);
  return st;
}

int mpspmv_mlp_grad(const float* params, int C, const float* X, const int* y, int B, float* grads, float* loss,
                    void* stream) {
  if (!params || !X || !y || !grads || B < 1 || C < 2 || C > 16) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  float* buf = nullptr;
  MlpWork w;
  int st = mlp_alloc(B, C, &buf, w);
  if (st) return st;
  const MlpView v = mlp_view(params, C);
  mlp_forward(v, X, B, C, w, s);
  mlp_backward(v, X, y, B, C, w, grads, s);
  std::vector<float> lb(B);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(lb.data(), w.loss, sizeof(float) * B, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    st = MPSPMV_ECUDA;
  cudaFree(buf);
  if (!st && loss) {
    double t = 0;
    for (float v2 : lb) t += v2;
    *loss = (float)(t / B);
  }
  return st;
}

int mpspmv_mlp_train(float* params, int C, const float* X, const int* y, int n, int batch, int epochs, float lr,
                     float* loss_per_epoch, void* stream) {
  if (!params || !X || !y || n < 1 || batch < 1 || epochs < 0 || C < 2 || C > 16 || !(lr > 0)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  const int B = std::min(batch, n);
  float* buf = nullptr;
  MlpWork w;
  int st = mlp_alloc(B, C, &buf, w);
  if (st) return st;
  float* g = nullptr;
  const int64_t np = mlp_param_count(C);
  if (cudaMalloc(&g, sizeof(float) * np) != cudaSuccess) {
    cudaFree(buf);
    return MPSPMV_ENOMEM;
  }
  const MlpView v = mlp_view(params, C);
  std::vector<float> lb(B);
  for (int ep = 0; ep < epochs && !st; ep++) {
    double tot = 0;
    int cnt = 0;
    // mini-batches in data order (the caller shuffles between calls)
    for (int b0 = 0; b0 + B <= n; b0 += B) {
      const float* Xb = X + (int64_t)b0 * D0;
      const int* yb = y + b0;
      mlp_forward(v, Xb, B, C, w, s);
      mlp_backward(v, Xb, yb, B, C, w, g, s);
      sgd_kernel<<<nb(np), kFT, 0, s>>>(params, g, np, lr);
      if (loss_per_epoch) {
        if (cudaMemcpyAsync(lb.data(), w.loss, sizeof(float) * B, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          st = MPSPMV_ECUDA;
          break;
        }
        for (float v2 : lb) tot += v2;
        cnt += B;
      }
    }
    if (cudaGetLastError() != cudaSuccess) st = MPSPMV_ECUDA;
    if (loss_per_epoch) loss_per_epoch[ep] = cnt ? (float)(tot / cnt) : 0.0f;
  }
  if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = MPSPMV_ECUDA;
  cudaFree(g);
  cudaFree(buf);
  return st;
}

int mpspmv_mlp_standardize(const float* X, int n, float* mu, float* sd, float* Xs, void* stream) {
  if (!X || !mu || !sd || !Xs || n < 1) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  standardize_kernel<<<1, D0, 0, s>>>(X, n, mu, sd, Xs);
  MPS_CUDA(cudaGetLastError());
  return MPSPMV_OK;
}

int mpspmv_mlp_fold(float* params, int C, const float* mu, const float* sd, void* stream) {
  if (!params || !mu || !sd || C < 2 || C > 16) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  const MlpView v = mlp_view(params, C);
  fold_kernel<<<1, D1, 0, s>>>(const_cast<float*>(v.W1), const_cast<float*>(v.b1), mu, sd);
  MPS_CUDA(cudaGetLastError());
  return MPSPMV_OK;
}

int mpspmv_features(mpspmv_h h, const double* cg_hist, float* feat, void* stream) {
  if (!h || !feat) return MPSPMV_EINVAL;
  return mps_features(h, cg_hist, feat, mps_stream(stream));
}

}  // extern "C"
