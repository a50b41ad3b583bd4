// Learned Davidson guess and diagonal preconditioner of libxs.
//
// Per orbital pair (i, a) among the lowest orbital-energy gaps, eleven features
// (gap, orbital energies, centroid distance, spreads, s characters, the
// one-centre self-overlap of the transition charge, the density overlap, and
// the Coulomb energy of the two orbital densities in the monopole picture,
// sum_AB q_A(i) (s_A s_A|s_B s_B) q_B(a)) feed
// an MLP (11 -> 256 -> 256 -> 256 -> 2, gelu, weights rounded to bfloat16,
// float32 accumulation) whose two outputs are
//   0: the diagonal shift d_ia = A_ia,ia - (eps_a - eps_i) = 2(ia|ia) - (ii|aa)
//      (used as the preconditioner r / (omega - d eps - d));
//   1: a score, log10 of the pair's weight sum_n X_n,ia^2 in the lowest roots
//      (used to pick the initial unit vectors).
// Training targets come from the exact diagonal (float64, two-centre part as
// P W P^T over packed pair densities plus closed-form one-centre terms) and
// from converged amplitudes.  Training and inference run through the
// project's own kernels (split-TF32 tensor-core GEMM, gelu, Adam); nothing here changes the
// converged roots: the plain Davidson judges the result.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "kernels.h"
#include "mlp.h"
#include "tc_gemm.h"

namespace xs {

namespace {

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// float -> nearest bfloat16 value (kept in a float), ties to even
__device__ __forceinline__ float round_bf16(float x) {
  uint32_t b = __float_as_uint(x);
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7FFFu + lsb;
  return __uint_as_float(b & 0xFFFF0000u);
}

__global__ void bias_act_kernel(int rows, int cols, float* Z, const float* __restrict__ bias, float* H, int act) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * cols) return;
  const int c = static_cast<int>(idx % cols);
  const float z = Z[idx] + bias[c];
  Z[idx] = z;
  H[idx] = act ? gelu_f(z) : z;
}

// dL/dY of the weighted mean-squared error; loss contributions summed into *loss
__global__ void mse_grad_kernel(int rows, int cols, const float* __restrict__ Y, const float* __restrict__ T,
                                const float* __restrict__ w, float* G, float* loss) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (idx < (long long)rows * cols) {
    const int c = static_cast<int>(idx % cols);
    const float d = Y[idx] - T[idx];
    const float scale = 1.0f / (float)((long long)rows * cols);
    G[idx] = 2.0f * d * w[c] * scale;
    l = d * d * w[c] * scale;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

__global__ void gelu_back_kernel(long long n, const float* __restrict__ Z, float* G) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) G[idx] *= gelu_grad_f(Z[idx]);
}

__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ G, float* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += G[(long long)r * cols + c];
  out[c] = s;
}

// Adam step on the float32 master weights; wq gets the bfloat16-rounded copy
__global__ void adam_kernel(int n, float* w, float* wq, const float* __restrict__ g, float* m, float* v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = b1 * m[i] + (1.0f - b1) * gi;
  v[i] = b2 * v[i] + (1.0f - b2) * gi * gi;
  w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
  wq[i] = round_bf16(w[i]);
}

__global__ void round_kernel(int n, const float* __restrict__ w, float* wq) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wq[i] = round_bf16(w[i]);
}

// per MO p: centroid (3), spread, s character from populations C_mu,p^2
__global__ void mo_stats_kernel(int n, const double* __restrict__ CT, const int* __restrict__ ao_atom,
                                const int* __restrict__ ao_local, const double* __restrict__ xyz, double* stats) {
  const int p = blockIdx.x;
  double c[3] = {0, 0, 0}, r2 = 0, s = 0;
  for (int mu = threadIdx.x; mu < n; mu += blockDim.x) {
    const double q = CT[(long long)p * n + mu] * CT[(long long)p * n + mu];
    const int A = ao_atom[mu];
    for (int x = 0; x < 3; ++x) c[x] += q * xyz[3 * A + x];
    r2 += q * (xyz[3 * A] * xyz[3 * A] + xyz[3 * A + 1] * xyz[3 * A + 1] + xyz[3 * A + 2] * xyz[3 * A + 2]);
    if (ao_local[mu] == 0) s += q;
  }
  __shared__ double red[5][32];
  double v[5] = {c[0], c[1], c[2], r2, s};
  for (int k = 0; k < 5; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double out[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k)
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) out[k] += red[k][j];
    const double spread2 = out[3] - (out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    stats[p * 6 + 0] = out[0];
    stats[p * 6 + 1] = out[1];
    stats[p * 6 + 2] = out[2];
    stats[p * 6 + 3] = sqrt(fmax(spread2, 0.0));
    stats[p * 6 + 4] = out[4];
  }
}

// features of the pairs (flattened ia = i * v + a)
__global__ void features_kernel(int npairs, int n, int o, int v, int natoms, const long long* __restrict__ pairs,
                                const double* __restrict__ CT, const double* __restrict__ eps,
                                const double* __restrict__ stats, const int* __restrict__ atom_ao_off,
                                const int* __restrict__ atom_nao, float* F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npairs) return;
  const int i = static_cast<int>(pairs[k] / v), a = o + static_cast<int>(pairs[k] % v);
  const double* si = stats + i * 6;
  const double* sa = stats + a * 6;
  const double dx = si[0] - sa[0], dy = si[1] - sa[1], dz = si[2] - sa[2];
  double tq2 = 0.0, ov = 0.0;
  for (int A = 0; A < natoms; ++A) {
    double t = 0.0, qi = 0.0, qa = 0.0;
    for (int u = 0; u < atom_nao[A]; ++u) {
      const int mu = atom_ao_off[A] + u;
      const double ci = CT[(long long)i * n + mu], ca = CT[(long long)a * n + mu];
      t += ci * ca;
      qi += ci * ci;
      qa += ca * ca;
    }
    tq2 += t * t;
    ov += qi * qa;
  }
  float* f = F + (long long)k * kMlpFeatures;
  f[0] = static_cast<float>((eps[a] - eps[i]) / 10.0);
  f[1] = static_cast<float>(eps[i] / 10.0);
  f[2] = static_cast<float>(eps[a] / 10.0);
  f[3] = static_cast<float>(sqrt(dx * dx + dy * dy + dz * dz) / 5.0);
  f[4] = static_cast<float>(si[3] / 5.0);
  f[5] = static_cast<float>(sa[3] / 5.0);
  f[6] = static_cast<float>(si[4]);
  f[7] = static_cast<float>(sa[4]);
  f[8] = static_cast<float>(tq2);
  f[9] = static_cast<float>(ov);
}

// atomic populations q[A][p] = sum_{mu on A} C_mu,p^2 (natoms x n)
// Mulliken-like atomic populations of every MO: qT[p][A] = sum_{u on A} C[u][p]^2
__global__ void populations_kernel(int n, int natoms, const double* __restrict__ CT,
                                   const int* __restrict__ atom_ao_off, const int* __restrict__ atom_nao, double* qT) {
  const int p = blockIdx.y;
  const int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= natoms) return;
  double s = 0.0;
  for (int u = 0; u < atom_nao[A]; ++u) {
    const double c = CT[(long long)p * n + atom_ao_off[A] + u];
    s += c * c;
  }
  qT[(long long)p * natoms + A] = s;
}

// monopole Coulomb matrix gamma_AB = (s_A s_A | s_B s_B), gamma_AA = gss_A
__global__ void gamma_kernel(int natoms, int np, const double* __restrict__ W, const int* __restrict__ atom_prod_off,
                             const int* __restrict__ atom_elem, const double* __restrict__ par, double* g) {
  const int A = blockIdx.y, B = blockIdx.x * blockDim.x + threadIdx.x;
  if (B >= natoms) return;
  g[(long long)A * natoms + B] = (A == B) ? par[atom_elem[A] * XS_NPARAM + 4]
                                          : W[(long long)atom_prod_off[A] * np + atom_prod_off[B]];
}

// monopole Coulomb energy of each pair's orbital densities, one warp per pair:
// J = sum_A qT[i][A] tT[a][A] with tT = q_vir^T gamma; feature 10 = J / 10
__global__ void pair_coulomb_kernel(int npairs, int o, int v, int natoms, const long long* __restrict__ pairs,
                                    const double* __restrict__ qT, const double* __restrict__ tT, float* F) {
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (k >= npairs) return;
  const long long pk = pairs[k];
  const int i = static_cast<int>(pk / v), a = static_cast<int>(pk % v);
  const double* qi = qT + (long long)i * natoms;
  const double* ta = tT + (long long)a * natoms;
  double sum = 0.0;
  for (int A = lane; A < natoms; A += 32) sum += qi[A] * ta[A];
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (lane == 0) F[(long long)k * kMlpFeatures + 10] = static_cast<float>(sum / 10.0);
}

__device__ __forceinline__ int pidx_m(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int base[4] = {0, 4, 7, 9};
  return base[lo] + (hi - lo);
}

// packed pair densities of the pairs: kind 0 rho^{ia}, 1 rho^{ii}, 2 rho^{aa}
__global__ void pack_pairs_kernel(int npairs, int n, int o, int v, int natoms, int np,
                                  const long long* __restrict__ pairs, const double* __restrict__ CT,
                                  const int* __restrict__ atom_ao_off, const int* __restrict__ atom_nao,
                                  const int* __restrict__ atom_prod_off, int kind, double* P) {
  const int k = blockIdx.y;
  const int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npairs || A >= natoms) return;
  const int i = static_cast<int>(pairs[k] / v), a = o + static_cast<int>(pairs[k] % v);
  const int p1 = (kind == 2) ? a : i, p2 = (kind == 1) ? i : a;
  const int off = atom_ao_off[A], na = atom_nao[A], PA = atom_prod_off[A];
  for (int u = 0; u < na; ++u)
    for (int w = u; w < na; ++w) {
      const double x = CT[(long long)p1 * n + off + u] * CT[(long long)p2 * n + off + w];
      const double y = CT[(long long)p1 * n + off + w] * CT[(long long)p2 * n + off + u];
      const int q = (na == 4) ? pidx_m(u, w) : 0;
      P[(long long)k * np + PA + q] = (u == w) ? x : x + y;
    }
}

// one-centre part of (p1 p2 | p3 p4) summed over atoms, closed-form integrals
__device__ double one_centre_quad(const double* par, int Ael, int na, const double* c1, const double* c2,
                                  const double* c3, const double* c4) {
  const double* pp = par + Ael * XS_NPARAM;
  const double gss = pp[4], gsp = pp[5], gpp = pp[6], gp2 = pp[7], hsp = pp[8], hpp = 0.5 * (gpp - gp2);
  if (na == 1) return gss * c1[0] * c2[0] * c3[0] * c4[0];
  // (mu nu | lam sig) of one heavy atom
  auto I = [&](int m, int nn, int l, int s) -> double {
    if (m == nn && l == s) {
      if (m == 0 && l == 0) return gss;
      if (m == 0 || l == 0) return gsp;
      return (m == l) ? gpp : gp2;
    }
    if (m != nn && l != s) {
      const bool same = (m == l && nn == s) || (m == s && nn == l);
      if (!same) return 0.0;
      return (m == 0 || nn == 0) ? hsp : hpp;
    }
    return 0.0;
  };
  double acc = 0.0;
  for (int m = 0; m < 4; ++m)
    for (int nn = 0; nn < 4; ++nn) {
      const double x = c1[m] * c2[nn];
      if (x == 0.0) continue;
      for (int l = 0; l < 4; ++l)
        for (int s = 0; s < 4; ++s) acc += x * I(m, nn, l, s) * c3[l] * c4[s];
    }
  return acc;
}

// shift = 2 (ia|ia) - (ii|aa): rowdot terms for the two-centre part plus one-centre sums
__global__ void diag_shift_kernel(int npairs, int n, int o, int v, int natoms, int np,
                                  const long long* __restrict__ pairs, const double* __restrict__ CT,
                                  const int* __restrict__ atom_ao_off, const int* __restrict__ atom_nao,
                                  const int* __restrict__ atom_elem, const double* __restrict__ par,
                                  const double* __restrict__ Pia, const double* __restrict__ Tia,
                                  const double* __restrict__ Pii, const double* __restrict__ Taa, double* shift) {
  const int k = blockIdx.x;
  const int i = static_cast<int>(pairs[k] / v), a = o + static_cast<int>(pairs[k] % v);
  double s1 = 0.0, s2 = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    s1 += Pia[(long long)k * np + p] * Tia[(long long)k * np + p];
    s2 += Pii[(long long)k * np + p] * Taa[(long long)k * np + p];
  }
  for (int A = threadIdx.x; A < natoms; A += blockDim.x) {
    double ci[4] = {0, 0, 0, 0}, ca[4] = {0, 0, 0, 0};
    const int na = atom_nao[A], off = atom_ao_off[A];
    for (int u = 0; u < na; ++u) {
      ci[u] = CT[(long long)i * n + off + u];
      ca[u] = CT[(long long)a * n + off + u];
    }
    s1 += one_centre_quad(par, atom_elem[A], na, ci, ca, ci, ca);
    s2 += one_centre_quad(par, atom_elem[A], na, ci, ci, ca, ca);
  }
  __shared__ double red[2][32];
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o2);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o2);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s1; red[1][threadIdx.x >> 5] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a1 = 0.0, a2 = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { a1 += red[0][j]; a2 += red[1][j]; }
    shift[k] = 2.0 * a1 - a2;
  }
}

}  // namespace

// ---- network -------------------------------------------------------------

int Mlp::nparams() const {
  int t = 0;
  for (int l = 0; l < kMlpLayers; ++l) t += sizes[l + 1] * sizes[l] + sizes[l + 1];
  return t;
}

void Mlp::init(cudaStream_t s, unsigned long long seed) {
  const int np_ = nparams();
  std::vector<float> h(np_, 0.0f);
  // weights uniform in +-1/sqrt(fan_in) from a 64-bit linear congruential stream, biases zero
  unsigned long long st = seed * 6364136223846793005ull + 1442695040888963407ull;
  int off = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    const int fin = sizes[l], fout = sizes[l + 1];
    const float lim = 1.0f / std::sqrt(static_cast<float>(fin));
    for (int k = 0; k < fout * fin; ++k) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      const double u = static_cast<double>(st >> 11) * (1.0 / 9007199254740992.0);
      h[off + k] = static_cast<float>((2.0 * u - 1.0) * lim);
    }
    off += fout * fin + fout;
  }
  set(s, h.data());
}

void Mlp::set(cudaStream_t s, const float* host) {
  const int np_ = nparams();
  w.alloc(np_);
  wq.alloc(np_);
  m.alloc(np_);
  v.alloc(np_);
  g.alloc(np_);
  XS_CUDA(cudaMemcpyAsync(w.get(), host, sizeof(float) * np_, cudaMemcpyHostToDevice, s));
  XS_CUDA(cudaMemsetAsync(m.get(), 0, sizeof(float) * np_, s));
  XS_CUDA(cudaMemsetAsync(v.get(), 0, sizeof(float) * np_, s));
  round_kernel<<<grid1(np_, 256), 256, 0, s>>>(np_, w.get(), wq.get());
  XS_CHECK_LAUNCH();
  step = 0;
  ready = true;
}

void Mlp::get(cudaStream_t s, float* host) const {
  XS_CUDA(cudaMemcpyAsync(host, w.get(), sizeof(float) * nparams(), cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
}

// activations: per layer Z (pre-activation) and H (output); H[-1] = input
namespace {

// D (M x N, row stride ldd) = A B^T on the tensor cores: A is M x K and B is
// N x K, each row-major with row stride ld, or given as its transpose (K x M,
// K x N) when ta / tb.  Both are split into TF32 pairs (hi + lo, the K padding
// zero; the bfloat16-rounded weights have lo = 0) and multiplied as
// hi*hi + hi*lo + lo*hi with float32 accumulation.
void tc_mm(cudaStream_t s, MlpOperands& w, int M, int N, int K, const float* A, int lda, bool ta, const float* B,
           int ldb, bool tb, float* D, int ldd) {
  if (!w.err.get()) {
    w.err.alloc(1);
    XS_CUDA(cudaMemsetAsync(w.err.get(), 0, sizeof(int), s));
  }
  const int Kp = pad32(K);
  w.ah.ensure((size_t)M * Kp);
  w.al.ensure((size_t)M * Kp);
  w.bh.ensure((size_t)N * Kp);
  w.bl.ensure((size_t)N * Kp);
  split_pad<float>(s, M, K, Kp, A, lda, 0, 0, 1, ta, w.ah.get(), w.al.get());
  split_pad<float>(s, N, K, Kp, B, ldb, 0, 0, 1, tb, w.bh.get(), w.bl.get());
  const TcOperand oa{w.ah.get(), w.al.get(), Kp, 0, false}, ob{w.bh.get(), w.bl.get(), Kp, 0, false};
  TcEpilogue e;
  e.mode = 0;
  e.D = D;
  e.ld = ldd;
  tc_gemm(s, oa, ob, M, N, Kp, 1, e, w.err.get());
}

}  // namespace

void Mlp::check(cudaStream_t s, MlpOperands& w) {
  if (!w.err.get()) return;
  int h = 0;
  XS_CUDA(cudaMemcpyAsync(&h, w.err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
  if (h) {
    XS_CUDA(cudaMemsetAsync(w.err.get(), 0, sizeof(int), s));
    throw Error(XS_ETIMEOUT, "network product: a bounded device wait timed out (code " + std::to_string(h) + ")");
  }
}

void Mlp::forward(cudaStream_t s, int rows, const float* X, std::vector<DevBuf<float>>& Z,
                  std::vector<DevBuf<float>>& H, MlpOperands& mo) const {
  Z.resize(kMlpLayers);
  H.resize(kMlpLayers);
  const float* in = X;
  int off = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    const int fin = sizes[l], fout = sizes[l + 1];
    Z[l].ensure((size_t)rows * fout);
    H[l].ensure((size_t)rows * fout);
    const float* W = wq.get() + off;
    const float* b = wq.get() + off + fout * fin;
    // Z = in W^T  (rows x fout)
    tc_mm(s, mo, rows, fout, fin, in, fin, false, W, fin, false, Z[l].get(), fout);
    bias_act_kernel<<<grid1((long long)rows * fout, 256), 256, 0, s>>>(rows, fout, Z[l].get(), b, H[l].get(),
                                                                      l < kMlpLayers - 1 ? 1 : 0);
    XS_CHECK_LAUNCH();
    in = H[l].get();
    off += fout * fin + fout;
  }
}

float Mlp::gradient(cudaStream_t s, int rows, const float* X, const float* T, const float* colw,
                   DevBuf<float>& scratch, MlpOperands& mo) {
  std::vector<DevBuf<float>> Z, H;
  forward(s, rows, X, Z, H, mo);
  const int nout = sizes[kMlpLayers];
  scratch.ensure((size_t)rows * kMlpHidden * 2 + 8);
  float* loss = scratch.get();
  float* G = scratch.get() + 8;
  float* G2 = G + (size_t)rows * kMlpHidden;
  XS_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  mse_grad_kernel<<<grid1((long long)rows * nout, 256), 256, 0, s>>>(rows, nout, H[kMlpLayers - 1].get(), T, colw, G,
                                                                     loss);
  XS_CHECK_LAUNCH();
  // offsets of each layer's block in the flat parameter vector
  std::vector<int> off(kMlpLayers + 1, 0);
  for (int l = 0; l < kMlpLayers; ++l) off[l + 1] = off[l] + sizes[l + 1] * sizes[l] + sizes[l + 1];
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const int fin = sizes[l], fout = sizes[l + 1];
    if (l < kMlpLayers - 1) {
      gelu_back_kernel<<<grid1((long long)rows * fout, 256), 256, 0, s>>>((long long)rows * fout, Z[l].get(), G);
      XS_CHECK_LAUNCH();
    }
    const float* hin = (l == 0) ? X : H[l - 1].get();
    // dW = G^T hin (fout x fin), db = column sums of G
    tc_mm(s, mo, fout, fin, rows, G, fout, true, hin, fin, true, g.get() + off[l], fin);
    colsum_kernel<<<grid1(fout, 128), 128, 0, s>>>(rows, fout, G, g.get() + off[l] + fout * fin);
    XS_CHECK_LAUNCH();
    if (l > 0) {
      // G_prev = G W  (rows x fin), with the bfloat16 weights of the forward pass
      tc_mm(s, mo, rows, fin, fout, G, fout, false, wq.get() + off[l], fin, true, G2, fin);
      std::swap(G, G2);
    }
  }
  float hl = 0.0f;
  XS_CUDA(cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
  check(s, mo);
  return hl;
}

float Mlp::train_step(cudaStream_t s, int rows, const float* X, const float* T, const float* colw, float lr,
                      DevBuf<float>& scratch, MlpOperands& mo) {
  const float l = gradient(s, rows, X, T, colw, scratch, mo);
  ++step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, static_cast<float>(step));
  const float c2 = 1.0f - std::pow(b2, static_cast<float>(step));
  const int np_ = nparams();
  adam_kernel<<<grid1(np_, 256), 256, 0, s>>>(np_, w.get(), wq.get(), g.get(), m.get(), v.get(), lr, b1, b2, 1e-8f, c1,
                                              c2);
  XS_CHECK_LAUNCH();
  return l;
}

// ---- features and targets ----------------------------------------------------

std::vector<long long> lowest_gaps(const std::vector<double>& eps, int o, int v, long long k) {
  // (gap, pair) for every pair without per-comparison index arithmetic; the k
  // smallest by selection (linear) and a sort of those k; ties by pair index
  const long long ov = (long long)o * v;
  k = std::min(k, ov);
  std::vector<std::pair<double, long long>> g((size_t)ov);
  for (int i = 0; i < o; ++i)
    for (int a = 0; a < v; ++a) g[(size_t)i * v + a] = {eps[o + a] - eps[i], (long long)i * v + a};
  if (k < ov) std::nth_element(g.begin(), g.begin() + k, g.end());
  std::sort(g.begin(), g.begin() + k);
  std::vector<long long> out((size_t)k);
  for (long long q = 0; q < k; ++q) out[(size_t)q] = g[(size_t)q].second;
  return out;
}

std::vector<long long> lowest_gap_pairs(Ctx& c, const DevMol& m, int npairs) {
  std::vector<double> eps(m.n);
  XS_CUDA(cudaMemcpyAsync(eps.data(), m.eps.get(), sizeof(double) * m.n, cudaMemcpyDeviceToHost, c.stream));
  XS_CUDA(cudaStreamSynchronize(c.stream));
  return lowest_gaps(eps, m.o, m.v, npairs);
}

void pair_features(Ctx& c, const DevMol& m, const std::vector<long long>& pairs, float* F_dev,
                   DevBuf<long long>& dpairs, FeatureWork& fw) {
  cudaStream_t s = c.stream;
  const int npairs = static_cast<int>(pairs.size());
  dpairs.ensure(npairs);
  XS_CUDA(cudaMemcpyAsync(dpairs.get(), pairs.data(), sizeof(long long) * npairs, cudaMemcpyHostToDevice, s));
  fw.stats.ensure((size_t)m.n * 6);
  mo_stats_kernel<<<m.n, 128, 0, s>>>(m.n, m.CT.get(), m.ao_atom.get(), m.ao_local.get(), m.xyz.get(),
                                      fw.stats.get());
  XS_CHECK_LAUNCH();
  features_kernel<<<grid1(npairs, 128), 128, 0, s>>>(npairs, m.n, m.o, m.v, m.L.natoms, dpairs.get(), m.CT.get(),
                                                     m.eps.get(), fw.stats.get(), m.atom_ao_off.get(),
                                                     m.atom_nao.get(), F_dev);
  XS_CHECK_LAUNCH();
  // monopole Coulomb energy of the orbital densities of each pair:
  // J_ia = q(i)^T Gamma q(a), q(p) the atomic populations of MO p
  const int N = m.L.natoms;
  fw.q.ensure((size_t)N * m.n);
  fw.gam.ensure((size_t)N * N);
  fw.t.ensure((size_t)N * m.v);
  populations_kernel<<<dim3((N + 127) / 128, m.n), 128, 0, s>>>(m.n, N, m.CT.get(), m.atom_ao_off.get(),
                                                               m.atom_nao.get(), fw.q.get());
  gamma_kernel<<<dim3((N + 127) / 128, N), 128, 0, s>>>(N, m.np, m.W.get(), m.atom_prod_off.get(), m.atom_elem.get(),
                                                        c.d_par.get(), fw.gam.get());
  XS_CHECK_LAUNCH();
  // tT (v x N) = q_vir^T Gamma (Gamma symmetric)
  gemm<double>(s, false, false, m.v, N, N, 1.0, fw.q.get() + (size_t)m.o * N, N, 0, fw.gam.get(), N, 0, 0.0,
               fw.t.get(), N, 0, 1);
  pair_coulomb_kernel<<<grid1((long long)npairs * 32, 256), 256, 0, s>>>(npairs, m.o, m.v, N, dpairs.get(),
                                                                        fw.q.get(), fw.t.get(), F_dev);
  XS_CHECK_LAUNCH();
}

void diagonal_shift(Ctx& c, const DevMol& m, const std::vector<long long>& pairs, double* shift_dev) {
  cudaStream_t s = c.stream;
  const int npairs = static_cast<int>(pairs.size());
  const int np = m.np;
  DevBuf<long long> dp(npairs);
  XS_CUDA(cudaMemcpyAsync(dp.get(), pairs.data(), sizeof(long long) * npairs, cudaMemcpyHostToDevice, s));
  DevBuf<double> Pia((size_t)npairs * np), Pii((size_t)npairs * np), Paa((size_t)npairs * np);
  DevBuf<double> Tia((size_t)npairs * np), Taa((size_t)npairs * np);
  dim3 grid((m.L.natoms + 127) / 128, npairs);
  pack_pairs_kernel<<<grid, 128, 0, s>>>(npairs, m.n, m.o, m.v, m.L.natoms, np, dp.get(), m.CT.get(),
                                         m.atom_ao_off.get(), m.atom_nao.get(), m.atom_prod_off.get(), 0, Pia.get());
  pack_pairs_kernel<<<grid, 128, 0, s>>>(npairs, m.n, m.o, m.v, m.L.natoms, np, dp.get(), m.CT.get(),
                                         m.atom_ao_off.get(), m.atom_nao.get(), m.atom_prod_off.get(), 1, Pii.get());
  pack_pairs_kernel<<<grid, 128, 0, s>>>(npairs, m.n, m.o, m.v, m.L.natoms, np, dp.get(), m.CT.get(),
                                         m.atom_ao_off.get(), m.atom_nao.get(), m.atom_prod_off.get(), 2, Paa.get());
  XS_CHECK_LAUNCH();
  // T = P W (W symmetric, zero diagonal atom blocks)
  gemm<double>(s, false, false, npairs, np, np, 1.0, Pia.get(), np, 0, m.W.get(), np, 0, 0.0, Tia.get(), np, 0, 1);
  gemm<double>(s, false, false, npairs, np, np, 1.0, Paa.get(), np, 0, m.W.get(), np, 0, 0.0, Taa.get(), np, 0, 1);
  diag_shift_kernel<<<npairs, 128, 0, s>>>(npairs, m.n, m.o, m.v, m.L.natoms, np, dp.get(), m.CT.get(),
                                           m.atom_ao_off.get(), m.atom_nao.get(), m.atom_elem.get(), c.d_par.get(),
                                           Pia.get(), Tia.get(), Pii.get(), Taa.get(), shift_dev);
  XS_CHECK_LAUNCH();
  XS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace xs
