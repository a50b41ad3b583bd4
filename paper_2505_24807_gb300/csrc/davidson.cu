// Davidson solver of libxs (paper, Section "GPU Implementation", batched
// steps 1-6), float64 subspace on the device:
//   1. orthonormal start V (unit vectors on the lowest orbital-energy gaps);
//   2. products A V (CIS) or (A+B) V, (A-B) V (TDHF);
//   3. projected matrices, kept incrementally (new columns per iteration), and
//      their diagonalisation by the Jacobi kernel; lowest k Ritz pairs;
//   4. Ritz vectors X = V x;
//   5. residuals r = A X - omega X and their norms; converged roots drop out;
//   6. diagonal preconditioner r / (omega - d eps), Gram-Schmidt twice against
//      V, Loewdin orthonormalisation of the new block, append.
// TDHF uses the symmetric subspace form of Stratmann, Scuseria and Frisch
// (J. Chem. Phys. 109, 8218 (1998)) -- the paper names Davidson for RPA
// without the variant: a- = V^T (A-B) V, M = a-^(1/2) a+ a-^(1/2), M z =
// omega^2 z, X+Y = V a-^(1/2) z / sqrt(omega), X-Y = V a+ (X+Y)~ / omega,
// residuals (A+B)(X+Y) - omega (X-Y) and (A-B)(X-Y) - omega (X+Y).
// When V would exceed max_subspace it collapses onto the current Ritz
// vectors (CIS: the 2k lowest; TDHF: span of X+Y and X-Y), the restart of
// the paper's Section "Results and discussion".
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "davidson.h"
#include "kernels.h"
#include "products.h"
#include "small.h"
#include "syev.h"
#include "mlp.h"
#include "ozaki.h"

namespace xs {

namespace {

constexpr double kLowdinThresh = 1e-14;
constexpr double kMixedResidualFloor = 1e-4;
// mixed solves of at least this many amplitudes run the float64 subspace
// products on the tensor cores (exact digit splitting)
constexpr long long kOzMinLength = 32768;
// learned guess: candidate pairs (the lowest orbital-energy gaps) that the
// network scores; its preconditioner shift covers these pairs
constexpr long long kLearnedPairs = 16384;

struct Work {
  DevBuf<double> V, S1, S2;        // Smax x ov
  DevBuf<double> a1, a2;           // Smax x Smax, upper part valid
  DevBuf<double> E, Q, w, E2, Q2, w2, Sh, tS;   // S x S work
  DevBuf<double> cu, cw;           // S x kk coefficient blocks
  DevBuf<double> X, U, Wv, PU, MW, R1, T;  // X: 2kk x ov (Ritz vectors, then X-Y or A X); R1: residual rows
  double* AX = nullptr;                          // = X + kk * ov
  DevBuf<double> C1, C2, C3;       // collapse scratch (2kk x ov)
  DevBuf<double> nrm, nrm2, omega, Bm;
  DevBuf<int> flag;
  DevBuf<long long> idx;
  DevBuf<double> gws, eig_ws;
  // float64-accurate tensor-core subspace products (exact digit splitting):
  // V as Gram operand (tn) and as combination operand (nn), A V / (A+B) V and
  // (A-B) V as combination operands, one scratch tn operand (new vectors)
  bool oz = false;
  long long Lp = 0, Pv = 0, Pb = 0;   // amplitudes per plane; plane capacities of Vtn and Btn
  int ldk = 0, bcap = 0;
  DevBuf<oz_t> Vtn, Vnn, S1nn, S2nn, Btn, Tnn;
  int ldkT = 0;
  DevBuf<int> eV, eS1, eS2, eB;
  // per-row max |x| (abs_hi) formed by the kernels that write the rows
  // (product epilogues, combinations, row scaling): the digit exponents need
  // no extra pass over the float64 rows
  DevBuf<unsigned int> mxV, mxS1, mxS2, mxT;
  DevBuf<double> coef, rcoef;   // combination coefficients; the deferred TDHF Ritz block
  OzWork ozw;
  // learned guess: features, network activations, predicted shift
  FeatureWork fw;
  DevBuf<float> F;
  DevBuf<long long> dpairs;
  std::vector<DevBuf<float>> Z, H;
  MlpOperands mo;   // the network's tensor-core operand pairs
  DevBuf<double> lshift, dsh, fdev;
  // page-locked host staging of the per-iteration read-back
  double* hpin = nullptr;
  size_t hpin_n = 0;
  double* host_stage(size_t count) {
    if (count > hpin_n) {
      if (hpin) cudaFreeHost(hpin);
      hpin = nullptr;
      hpin_n = 0;
      XS_CUDA(cudaMallocHost(&hpin, sizeof(double) * count));
      hpin_n = count;
    }
    return hpin;
  }
  Work() = default;
  Work(const Work&) = delete;
  Work& operator=(const Work&) = delete;
  ~Work() { if (hpin) cudaFreeHost(hpin); }
};

// exponents of count rows of X: from the maxima the writing kernel formed
// (mx), else by a pass over the rows
void exponents(Ctx& c, Work& w, long long ov, const double* X, int count, int* e, const unsigned int* mx) {
  if (mx) oz_exponents_from_max(c.stream, count, mx, e, c.tc_err.get());
  else oz_exponents(c.stream, count, ov, X, ov, e, w.ozw, c.tc_err.get());
}

// digits of V rows [first, first + count) in both layouts (mx: their maxima, or null)
void slice_V(Ctx& c, Work& w, long long ov, int first, int count, const unsigned int* mx = nullptr) {
  if (!w.oz || count <= 0) return;
  const double* X = w.V.get() + (size_t)first * ov;
  exponents(c, w, ov, X, count, w.eV.get() + first, mx);
  oz_slice(c.stream, count, ov, X, ov, w.eV.get() + first, w.Vtn.get(), w.Pv, first, w.Vnn.get(), w.ldk, first);
}

// digits of product rows [first, first + count) (S1 or S2): nn layout, and the
// tn layout into rows tn_r0.. of the scratch operand Btn when with_tn
void slice_P(Ctx& c, Work& w, long long ov, const double* P, DevBuf<int>& e, DevBuf<oz_t>& nn, int first, int count,
             bool with_tn, int tn_r0 = 0, const unsigned int* mx = nullptr) {
  if (!w.oz || count <= 0) return;
  if (with_tn && tn_r0 + count > w.bcap) throw Error(XS_EINVAL, "subspace scratch operand too small");
  const double* X = P + (size_t)first * ov;
  exponents(c, w, ov, X, count, e.get() + first, mx);
  oz_slice(c.stream, count, ov, X, ov, e.get() + first, with_tn ? w.Btn.get() : nullptr, w.Pb, tn_r0, nn.get(),
           w.ldk, first);
}

// digits of count scratch rows T into Btn (exponents eB), and into Tnn when with_nn
void slice_T(Ctx& c, Work& w, long long ov, const double* T, int count, bool with_nn = false,
             const unsigned int* mx = nullptr) {
  if (count > w.bcap || (with_nn && count * kOzDigits > w.ldkT))
    throw Error(XS_EINVAL, "subspace scratch operand too small");
  exponents(c, w, ov, T, count, w.eB.get(), mx);
  oz_slice(c.stream, count, ov, T, ov, w.eB.get(), w.Btn.get(), w.Pb, 0, with_nn ? w.Tnn.get() : nullptr, w.ldkT, 0);
}

// Coefficients of the CIS step, outputs [X (kk) | R (kk)] with X_j = V q_j and
// R_j = A V q_j - omega_j V q_j; blocks (A V, V), S x 2kk each.
__global__ void cis_coef_kernel(int S, int k, int kk, const double* __restrict__ Q, int ldq,
                                const double* __restrict__ omega, double* __restrict__ out) {
  const int w2 = 2 * kk;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * w2) return;
  const int m = idx / w2, j = idx % w2;
  const int r = j < kk ? j : j - kk;
  const double q = r < k ? Q[(size_t)m * ldq + r] : 0.0;
  out[idx] = j < kk ? 0.0 : q;
  out[(size_t)S * w2 + idx] = j < kk ? q : (r < k ? -omega[r] * q : 0.0);
}

// Coefficients of the TDHF step: residual outputs [r1 (kk) | r2 (kk)] over the
// blocks ((A+B) V, V, (A-B) V) with r1_j = (A+B) V cu_j - omega_j V cw_j and
// r2_j = (A-B) V cw_j - omega_j V cu_j, then a fourth block for the Ritz
// vectors [V cu (kk) | V cw (kk)] over V; S x 2kk each.
__global__ void rpa_coef_kernel(int S, int k, int kk, const double* __restrict__ cu, const double* __restrict__ cw,
                                const double* __restrict__ omega, double* __restrict__ out) {
  const int w2 = 2 * kk;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * w2) return;
  const int m = idx / w2, j = idx % w2;
  const int r = j < kk ? j : j - kk;
  const bool ok = r < k;
  const double u = ok ? cu[(size_t)m * k + r] : 0.0;
  const double wv = ok ? cw[(size_t)m * k + r] : 0.0;
  const double om = ok ? omega[r] : 0.0;
  const size_t blk = (size_t)S * w2;
  out[idx] = j < kk ? u : 0.0;
  out[blk + idx] = j < kk ? -om * wv : -om * u;
  out[2 * blk + idx] = j < kk ? 0.0 : wv;
  out[3 * blk + idx] = j < kk ? u : wv;
}

void sync_copy(cudaStream_t s, void* dst, const void* src, size_t bytes) {
  // a copy into pageable host memory waits for the stream inside the copy call
  HostScope h_wait("host:sync_wait");
  XS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  XS_CUDA(cudaStreamSynchronize(s));
}

// nrm2[r] = 1 / nrm[r] (0 for a zero row)
__global__ void inv_norms_kernel(int n, const double* __restrict__ nrm, double* __restrict__ inv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) inv[r] = nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0;
}

// Orthonormalise the nnew rows of T against V[0:S] (classical Gram-Schmidt,
// repeated when the first pass cancels much of a row) and among themselves (Loewdin, dropping directions whose Gram
// eigenvalue is below kLowdinThresh); writes the kept rows to Vout (and,
// on the tensor-core subspace, their maxima to vmax when given).
int orthonormalise_append(Ctx& c, Work& w, int S, int nnew, long long ov, double* Vout,
                          unsigned int* vmax = nullptr) {
  cudaStream_t s = c.stream;
  // maxima of T's rows from the kernels that write them (tensor-core subspace)
  unsigned int* tmax = w.oz ? w.mxT.get() : nullptr;
  // unit rows first (on the device: no host round trip)
  row_norms(s, nnew, ov, w.T.get(), w.nrm.get());
  inv_norms_kernel<<<grid1(nnew, 64), 64, 0, s>>>(nnew, w.nrm.get(), w.nrm2.get());
  XS_CHECK_LAUNCH();
  scale_rows(s, nnew, ov, w.T.get(), w.nrm2.get(), tmax);
  std::vector<double> h(nnew);
  for (int pass = 0; pass < 2 && S > 0; ++pass) {
    if (w.oz) {
      slice_T(c, w, ov, w.T.get(), nnew, false, tmax);
      oz_gram(s, S, nnew, ov, w.Vtn.get(), w.Pv, w.eV.get(), w.Btn.get(), w.Pb, w.eB.get(), 1.0, 0.0, w.tS.get(),
              nnew, w.ozw, c.tc_err.get());
      const OzBlock b{w.Vnn.get(), w.ldk, w.eV.get(), w.tS.get(), nnew};
      oz_combine(s, 1, &b, S, nnew, ov, -1.0, 1.0, w.T.get(), ov, w.ozw, c.tc_err.get(), tmax);
    } else {
      gram<double>(s, S, nnew, static_cast<int>(ov), w.V.get(), static_cast<int>(ov), w.T.get(),
                   static_cast<int>(ov), w.tS.get(), nnew, 1.0, 0.0, w.gws);
      gemm<double>(s, true, false, nnew, static_cast<int>(ov), S, -1.0, w.tS.get(), nnew, 0, w.V.get(),
                   static_cast<int>(ov), 0, 1.0, w.T.get(), static_cast<int>(ov), 0, 1);
    }
    if (pass == 0) {
      // a second pass only when the first removed a large part of some row
      // (norm below 0.7 of the unit input): "twice is enough" criterion
      row_norms(s, nnew, ov, w.T.get(), w.nrm.get());
      sync_copy(s, h.data(), w.nrm.get(), sizeof(double) * nnew);
      if (*std::min_element(h.begin(), h.end()) >= 0.7) break;
    }
  }
  if (w.oz) {
    slice_T(c, w, ov, w.T.get(), nnew, true, tmax);
    oz_gram(s, nnew, nnew, ov, w.Btn.get(), w.Pb, w.eB.get(), w.Btn.get(), w.Pb, w.eB.get(), 1.0, 0.0, w.E2.get(),
            nnew, w.ozw, c.tc_err.get());
  } else {
    gram<double>(s, nnew, nnew, static_cast<int>(ov), w.T.get(), static_cast<int>(ov), w.T.get(),
                 static_cast<int>(ov), w.E2.get(), nnew, 1.0, 0.0, w.gws);
  }
  // Gram matrices of nearly dependent directions have eigenvalues spread over
  // many decades; two-sided Jacobi resolves the small ones to high relative
  // accuracy, which the Loewdin factors 1/sqrt(lambda) need
  jacobi_eig(s, nnew, w.E2.get(), nnew, w.Q2.get(), nnew, w.w2.get(), w.flag.get() + 1);
  lowdin(s, nnew, w.w2.get(), w.Q2.get(), nnew, kLowdinThresh, w.Bm.get(), nnew, w.flag.get() + 2);
  int nkeep = 0;
  sync_copy(s, &nkeep, w.flag.get() + 2, sizeof(int));
  if (nkeep > 0) {
    if (w.oz) {
      // Vout = Bm T on the tensor cores: coefficients Bm^T (nnew x nkeep)
      transpose(s, nkeep, nnew, w.Bm.get(), w.coef.get());
      const OzBlock b{w.Tnn.get(), w.ldkT, w.eB.get(), w.coef.get(), nkeep};
      oz_combine(s, 1, &b, nnew, nkeep, ov, 1.0, 0.0, Vout, ov, w.ozw, c.tc_err.get(), vmax);
    } else {
      gemm<double>(s, false, false, nkeep, static_cast<int>(ov), nnew, 1.0, w.Bm.get(), nnew, 0, w.T.get(),
                   static_cast<int>(ov), 0, 0.0, Vout, static_cast<int>(ov), 0, 1);
    }
  }
  return nkeep;
}

// guess: unit vectors on the nguess lowest eps_a - eps_i (ties: lower i, then a),
// or on the given pair list (learned guess)
void make_guess(Ctx& c, const DevMol& m, Work& w, int nguess, long long ov, const std::vector<long long>* chosen) {
  cudaStream_t s = c.stream;
  std::vector<long long> order;
  if (chosen) {
    order = *chosen;
  } else {
    std::vector<double> eps(m.n);
    sync_copy(s, eps.data(), m.eps.get(), sizeof(double) * m.n);
    order = lowest_gaps(eps, m.o, m.v, nguess);
  }
  XS_CUDA(cudaMemsetAsync(w.V.get(), 0, sizeof(double) * nguess * ov, s));
  w.idx.ensure(nguess);
  XS_CUDA(cudaMemcpyAsync(w.idx.get(), order.data(), sizeof(long long) * nguess, cudaMemcpyHostToDevice, s));
  unit_vectors(s, nguess, ov, w.idx.get(), w.V.get());
}

// Transition dipoles through the MO dipole integrals D^x_ia = <i|r_x|a>
// (paper, Section "Results": oscillator strengths of the excited states):
// the AO dipole operator is R_A on the diagonal plus the one-centre
// <s|r_x|p_x> = D1 of each heavy atom, so D^x = C_occ^T (r_x C_vir) with
// r_x C_vir formed elementwise; then d_n = sqrt(2) sum_ia U_n,ia D_ia and
// f_n = 2/3 omega_n |d_n|^2 in atomic units.

// Bt[a][mu] = (r_x C_vir)[mu][a], component x
__global__ void dipole_rc_kernel(int n, int o, int v, int x, const int* __restrict__ ao_atom,
                                 const int* __restrict__ ao_local, const int* __restrict__ atom_elem,
                                 const double* __restrict__ xyz, const double* __restrict__ par,
                                 const double* __restrict__ CT, double* __restrict__ Bt) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)v * n) return;
  const int a = static_cast<int>(idx / n), mu = static_cast<int>(idx % n);
  const int A = ao_atom[mu];
  const double* c = CT + (size_t)(o + a) * n;
  double r = xyz[3 * A + x] * c[mu];
  const int loc = ao_local[mu];
  const bool heavy = (loc == 0) ? (mu + 3 < n && ao_atom[mu + 3] == A && ao_local[mu + 3] == 3) : (loc > 0);
  if (heavy) {
    const double D1 = par[atom_elem[A] * XS_NPARAM + 9];
    if (loc == 0) r = fma(D1, c[mu + 1 + x], r);
    else if (loc == 1 + x) r = fma(D1, c[mu - 1 - x], r);
  }
  Bt[idx] = r;
}

__global__ void osc_from_dipoles_kernel(int k, const double* __restrict__ dm, const double* __restrict__ omega,
                                        double* __restrict__ f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s2 = 0.0;
  for (int x = 0; x < 3; ++x) {
    const double d = dm[j * 3 + x] * (1.4142135623730951 / kBohrA);
    s2 += d * d;
  }
  f[j] = (2.0 / 3.0) * (omega[j] / kHartreeEV) * s2;
}

}  // namespace

void mo_dipoles(Ctx& c, DevMol& m) {
  if (m.dip.get()) return;
  cudaStream_t s = c.stream;
  const int n = m.n, o = m.o, v = m.v;
  const long long ov = (long long)o * v;
  m.dip.alloc((size_t)3 * ov);
  c.ws4.ensure((size_t)v * n);
  for (int x = 0; x < 3; ++x) {
    dipole_rc_kernel<<<grid1((long long)v * n, 256), 256, 0, s>>>(n, o, v, x, m.ao_atom.get(), m.ao_local.get(),
                                                                m.atom_elem.get(), m.xyz.get(), c.d_par.get(),
                                                                m.CT.get(), c.ws4.get());
    XS_CHECK_LAUNCH();
    gemm<double>(s, false, true, o, v, n, 1.0, m.CT.get(), n, 0, c.ws4.get(), n, 0, 0.0, m.dip.get() + (size_t)x * ov, v,
                 0, 1);
  }
}

void oscillator_strengths(Ctx& c, DevMol& m, int kk, const double* U, const double* omega_dev, double* f_dev) {
  cudaStream_t s = c.stream;
  const long long ov = (long long)m.o * m.v;
  mo_dipoles(c, m);
  c.ws5.ensure((size_t)3 * kk);
  // dm[j][x] = sum_ia U_j,ia D^x_ia
  gram<double>(s, kk, 3, static_cast<int>(ov), U, static_cast<int>(ov), m.dip.get(), static_cast<int>(ov), c.ws5.get(),
               3, 1.0, 0.0, c.ws0);
  osc_from_dipoles_kernel<<<grid1(kk, 64), 64, 0, s>>>(kk, c.ws5.get(), omega_dev, f_dev);
  XS_CHECK_LAUNCH();
}

int davidson(Ctx& c, DevMol& m, const xs_ex_opts& opt, SolveStats& st) {
  using clk = std::chrono::steady_clock;
  cudaStream_t s = c.stream;
  const int o = m.o, v = m.v;
  const long long ov = (long long)o * v;
  const bool rpa = opt.method == XS_TDHF;
  const bool triplet = opt.spin == XS_TRIPLET;
  const int kk = static_cast<int>(std::min<long long>(opt.nroots, ov));
  const bool use_oz = opt.subspace == XS_SUBSPACE_EMULATED ||
                      (opt.subspace == XS_SUBSPACE_AUTO && opt.precision == XS_MIXED && ov >= kOzMinLength);
  // subspace cap: 10 vectors per root; TDHF 16 with the float64-pipe
  // subspace, and 20 with the tensor-core subspace on problems of at least
  // 2^19 amplitudes, where one product costs far more than the S^3 subspace
  // eigensolve (2200 AOs, 10 roots, learned guess: cap 200 vs 100 is 38 vs 55
  // iterations, 462 vs 484 ms; cap 240 is slower again).  Medium problems keep
  // 10: there the eigensolve is a third of the solve.
  const int per_root = !rpa ? 10 : (!use_oz ? 16 : (ov >= (1LL << 19) ? 20 : 10));
  int Smax = opt.max_subspace > 0 ? opt.max_subspace : std::max(48, per_root * kk);
  Smax = static_cast<int>(std::min<long long>(Smax, ov));
  Smax = std::min(Smax, 1000);
  const int max_iter = opt.max_iter > 0 ? opt.max_iter : 200;
  const int nguess = static_cast<int>(std::min<long long>(ov, std::max(2 * kk, kk + 2)));
  const int Smin = static_cast<int>(std::min<long long>(ov, nguess + 2 * kk));
  if (Smax < nguess + (rpa ? 2 : 1) * kk) Smax = Smin;
  const int maxnew = rpa ? 2 * kk : kk;
  // memory bound on the subspace: V and its products in float64 (and their
  // digit operands for the tensor-core subspace) take per_vec bytes per
  // stored vector; the cap is lowered to fit the budget (more restarts, same
  // roots), and a budget below the guess block plus one new block is an error
  {
    const double nstore = rpa ? 3.0 : 2.0;
    const double per_vec = 8.0 * nstore * ov + (use_oz ? 16.0 * (double)oz_lp(ov) + 16.0 * nstore * ov : 0.0);
    double budget = opt.memory_limit;
    if (!(budget > 0.0)) {
      size_t free_b = 0, total_b = 0;
      XS_CUDA(cudaMemGetInfo(&free_b, &total_b));
      double held = 0.0;   // this context's subspace buffers are reused
      if (c.dav_cache) {
        const Work& w0 = *static_cast<const Work*>(c.dav_cache.get());
        held = 8.0 * (double)(w0.V.n + w0.S1.n + w0.S2.n) + 2.0 * (double)(w0.Vtn.n + w0.Vnn.n + w0.S1nn.n + w0.S2nn.n);
      }
      // reserve: Ritz vectors, residuals, new directions and their digit
      // scratch (a few 2k-row blocks of amplitudes), product scratch, headroom
      const double reserve = 8.0 * ov * (8.0 * kk + 8.0) + 32.0 * ov * (2.0 * kk + 2.0) + 4.0 * 1073741824.0;
      budget = (double)free_b + held - reserve;
    }
    const double cap = std::floor(budget / per_vec);
    if (cap < Smin)
      throw Error(XS_ENOMEM, "subspace needs " + std::to_string(static_cast<long long>(Smin * per_vec)) +
                                 " bytes for its first " + std::to_string(Smin) + " vectors; budget " +
                                 std::to_string(static_cast<long long>(budget)));
    if (cap < Smax) Smax = static_cast<int>(cap);
  }
  st.smax = Smax;
  // Mixed-precision products carry rounding noise of ~1e-6 relative, so their
  // residuals cannot fall much below 1e-5 eV; the energies, quadratic in the
  // residual, are still converged far below 1e-5 eV at a 1e-4 eV residual.
  const double tol_eff = (opt.precision == XS_MIXED) ? std::max(opt.tol, kMixedResidualFloor) : opt.tol;
  st.tol_used = tol_eff;

  HostScope h_setup("host:setup");
  // the workspace persists in the context between solves (buffers only grow):
  // repeated solves of similar molecules allocate nothing
  if (!c.dav_cache) c.dav_cache = std::shared_ptr<void>(new Work(), [](void* p) { delete static_cast<Work*>(p); });
  Work& w = *static_cast<Work*>(c.dav_cache.get());
  w.V.ensure((size_t)Smax * ov);
  w.S1.ensure((size_t)Smax * ov);
  if (rpa) w.S2.ensure((size_t)Smax * ov);
  w.a1.ensure((size_t)Smax * Smax);
  if (rpa) w.a2.ensure((size_t)Smax * Smax);
  // small matrices: S x S subspace work and up to 2k x 2k blocks (tiny molecules can have Smax < 2k)
  const size_t SB = (size_t)std::max(Smax, 2 * kk + 2);
  const size_t SS = SB * SB;
  w.E.ensure(SS); w.Q.ensure(SS); w.w.ensure(SB); w.Sh.ensure(SS);
  w.tS.ensure(std::max(SS, (size_t)Smax * (4 * kk + 4)));   // also the S x 2 new-block TDHF projections
  w.E2.ensure(SS); w.Q2.ensure(SS); w.w2.ensure(SB);
  w.cu.ensure((size_t)Smax * 2 * kk); w.cw.ensure((size_t)Smax * kk);
  w.X.ensure((size_t)2 * kk * ov); w.R1.ensure((size_t)(rpa ? 2 : 1) * kk * ov);
  w.AX = w.X.get() + (size_t)kk * ov;
  w.T.ensure((size_t)maxnew * ov);
  if (rpa) w.MW.ensure((size_t)kk * ov);
  // residual rows: R1 (CIS: A X - omega X; TDHF: r1), R2 (TDHF: r2)
  double* R1p = w.R1.get();
  double* R2p = rpa ? w.R1.get() + (size_t)kk * ov : nullptr;
  w.oz = use_oz;
  if (w.oz) {
    if (!c.tc_err.get()) {
      c.tc_err.ensure(1);
      XS_CUDA(cudaMemsetAsync(c.tc_err.get(), 0, sizeof(int), s));
    }
    w.Lp = oz_lp(ov);
    w.Pv = (long long)Smax * kOzDigits;
    w.ldk = oz_ldk(Smax);
    const int tcap = std::max(maxnew, std::max(nguess, 2 * kk));   // rows of a new block
    w.bcap = (rpa ? 2 : 1) * tcap;                                  // TDHF projections: two blocks
    w.Vtn.ensure((size_t)Smax * kOzDigits * w.Lp);
    w.Btn.ensure((size_t)w.bcap * kOzDigits * w.Lp);
    w.Pb = (long long)w.bcap * kOzDigits;
    w.ldkT = oz_ldk(tcap);
    // digit rows past the live vectors are read (times zero coefficients) and
    // must be finite: zero them when (re)allocated; later contents are digits
    auto ensure_zeroed = [&](DevBuf<oz_t>& b, size_t count) {
      const oz_t* before = b.get();
      b.ensure(count);
      if (b.get() != before) XS_CUDA(cudaMemsetAsync(b.get(), 0, sizeof(oz_t) * b.n, s));
    };
    ensure_zeroed(w.Tnn, (size_t)ov * w.ldkT);
    ensure_zeroed(w.Vnn, (size_t)ov * w.ldk);
    ensure_zeroed(w.S1nn, (size_t)ov * w.ldk);
    if (rpa) ensure_zeroed(w.S2nn, (size_t)ov * w.ldk);
    w.eV.ensure(Smax); w.eS1.ensure(Smax); w.eS2.ensure(Smax); w.eB.ensure(w.bcap);
    w.mxV.ensure(Smax); w.mxS1.ensure(Smax); w.mxS2.ensure(Smax); w.mxT.ensure(w.bcap);
    w.coef.ensure((size_t)4 * Smax * 2 * kk);
    if (rpa) w.rcoef.ensure((size_t)Smax * 2 * kk);
  }
  w.nrm.ensure(2 * kk + 2); w.nrm2.ensure(2 * kk + 2); w.omega.ensure(kk); w.Bm.ensure(4 * kk * kk + 4);
  w.flag.ensure(4);
  XS_CUDA(cudaMemsetAsync(w.flag.get(), 0, 4 * sizeof(int), s));

  int prod_prec = opt.precision;
  std::vector<double> hw(kk), hn(2 * kk);
  // products timed by CUDA events on the stream (read once at the end)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prod_events;
  struct EventsGuard {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& ev;
    ~EventsGuard() {
      for (auto& e : ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    }
  } events_guard{prod_events};
  bool prod_max = false;   // the last products formed their rows' maxima
  auto apply = [&](int first, int count) {
    cudaEvent_t e0, e1;
    XS_CUDA(cudaEventCreate(&e0));
    XS_CUDA(cudaEventCreate(&e1));
    prod_events.emplace_back(e0, e1);
    XS_CUDA(cudaEventRecord(e0, s));
    // the tensor-core products' epilogue forms the rows' maxima for the digit split
    prod_max = w.oz && prod_prec == XS_MIXED;
    products(c, m, opt.method, prod_prec, count, w.V.get() + first * ov, w.S1.get() + first * ov,
             rpa ? w.S2.get() + first * ov : nullptr, triplet, prod_max ? w.mxS1.get() + first : nullptr,
             prod_max && rpa ? w.mxS2.get() + first : nullptr);
    XS_CUDA(cudaEventRecord(e1, s));
    st.products += count;
  };
  // read-back staging (page-locked, kept in the workspace): omega, norms, status words
  double* const hs = w.host_stage(3 * (size_t)kk + 8);
  // read back omega (k), residual norms (nn) and the status words in one synchronisation
  auto fetch = [&](int k, int nn) {
    XS_CUDA(cudaMemcpyAsync(hs, w.omega.get(), sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    XS_CUDA(cudaMemcpyAsync(hs + kk, w.nrm.get(), sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
    XS_CUDA(cudaMemcpyAsync(hs + 3 * kk, w.flag.get() + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (c.tc_err.get())
      XS_CUDA(cudaMemcpyAsync(hs + 3 * kk + 1, c.tc_err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    else
      std::memset(hs + 3 * kk + 1, 0, sizeof(double));
    {
      HostScope h_wait("host:fetch_wait");
      XS_CUDA(cudaStreamSynchronize(s));
    }
    std::copy(hs, hs + k, hw.begin());
    std::copy(hs + kk, hs + kk + nn, hn.begin());
    int flag3 = 0, tcerr = 0;
    std::memcpy(&flag3, hs + 3 * kk, sizeof(int));
    std::memcpy(&tcerr, hs + 3 * kk + 1, sizeof(int));
    return std::make_pair(flag3, tcerr);
  };

  // learned guess and diagonal shift: MLP outputs on the lowest-gap pairs
  const double* shift = nullptr;
  std::vector<long long> learned_pairs;
  // (the network was trained on singlet roots and shifts: triplets take the plain guess)
  if (opt.guess == XS_GUESS_LEARNED && !triplet && c.mlp && c.mlp->ready) {
    HostScope h_learned("host:learned_guess");
    const int npairs = static_cast<int>(std::min<long long>(ov, kLearnedPairs));
    std::vector<long long> pairs = lowest_gap_pairs(c, m, npairs);
    w.F.ensure((size_t)pairs.size() * kMlpFeatures);
    pair_features(c, m, pairs, w.F.get(), w.dpairs, w.fw);
    c.mlp->forward(s, static_cast<int>(pairs.size()), w.F.get(), w.Z, w.H, w.mo);
    std::vector<float> out(pairs.size() * kMlpOutputs);
    sync_copy(s, out.data(), w.H[kMlpLayers - 1].get(), sizeof(float) * out.size());
    Mlp::check(s, w.mo);
    // preconditioner shift on the candidate pairs, zero elsewhere
    std::vector<double> sh(pairs.size());
    for (size_t q = 0; q < pairs.size(); ++q) sh[q] = out[q * kMlpOutputs];
    w.lshift.ensure((size_t)ov);
    XS_CUDA(cudaMemsetAsync(w.lshift.get(), 0, sizeof(double) * ov, s));
    w.dsh.ensure(sh.size());
    XS_CUDA(cudaMemcpyAsync(w.dsh.get(), sh.data(), sizeof(double) * sh.size(), cudaMemcpyHostToDevice, s));
    scatter(s, static_cast<int>(pairs.size()), w.dpairs.get(), w.dsh.get(), w.lshift.get());
    shift = w.lshift.get();
    // guess: the pairs with the highest predicted weight in the low roots
    std::vector<size_t> idx(pairs.size());
    std::iota(idx.begin(), idx.end(), size_t(0));
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
      return out[x * kMlpOutputs + 1] > out[y * kMlpOutputs + 1];
    });
    for (int q = 0; q < nguess; ++q) learned_pairs.push_back(pairs[idx[q]]);
    st.learned = true;
  }
  make_guess(c, m, w, nguess, ov, learned_pairs.empty() ? nullptr : &learned_pairs);
  std::vector<double> max_res_hist;
  int S = nguess, Sold = 0;
  slice_V(c, w, ov, 0, S);
  apply(0, S);

  h_setup.stop();
  HostScope h_loop("host:loop");
  std::vector<char> conv(kk, 0);
  int it = 0, kq = 1;
  bool converged = false, polishing = false;
  int status = XS_OK;
  // TDHF on the tensor-core subspace: the Ritz vectors [X+Y; X-Y] = V [u~ w~]
  // are needed only when the solve ends, the polish starts or V is collapsed,
  // so their combination (one pass over V's digits) waits until then; the
  // coefficients of the last Rayleigh-Ritz step and the rows of V they refer
  // to (unchanged until a collapse) are kept
  bool ritz_pending = false;
  int ritz_S = 0;
  auto flush_ritz = [&]() {
    if (!ritz_pending) return;
    const OzBlock rz{w.Vnn.get(), w.ldk, w.eV.get(), w.rcoef.get(), 2 * kk};
    oz_combine(s, 1, &rz, ritz_S, 2 * kk, ov, 1.0, 0.0, w.X.get(), ov, w.ozw, c.tc_err.get());
    ritz_pending = false;
  };
  for (it = 1; it <= max_iter + 1; ++it) {
    // projected matrices: new columns Sold..S-1 over all rows 0..S-1
    if (w.oz) {
      const int cnt = S - Sold;
      slice_P(c, w, ov, w.S1.get(), w.eS1, w.S1nn, Sold, cnt, true, 0, prod_max ? w.mxS1.get() + Sold : nullptr);
      if (!rpa) {
        oz_gram(s, S, cnt, ov, w.Vtn.get(), w.Pv, w.eV.get(), w.Btn.get(), w.Pb, w.eS1.get() + Sold, 1.0, 0.0,
                w.a1.get() + Sold, Smax, w.ozw, c.tc_err.get());
      } else {
        // V^T [(A+B) V_new | (A-B) V_new] in one pass over V's digits
        slice_P(c, w, ov, w.S2.get(), w.eS2, w.S2nn, Sold, cnt, true, cnt, prod_max ? w.mxS2.get() + Sold : nullptr);
        XS_CUDA(cudaMemcpyAsync(w.eB.get(), w.eS1.get() + Sold, sizeof(int) * cnt, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpyAsync(w.eB.get() + cnt, w.eS2.get() + Sold, sizeof(int) * cnt, cudaMemcpyDeviceToDevice,
                                s));
        oz_gram(s, S, 2 * cnt, ov, w.Vtn.get(), w.Pv, w.eV.get(), w.Btn.get(), w.Pb, w.eB.get(), 1.0, 0.0, w.tS.get(),
                2 * cnt, w.ozw, c.tc_err.get());
        XS_CUDA(cudaMemcpy2DAsync(w.a1.get() + Sold, sizeof(double) * Smax, w.tS.get(), sizeof(double) * 2 * cnt,
                                  sizeof(double) * cnt, S, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpy2DAsync(w.a2.get() + Sold, sizeof(double) * Smax, w.tS.get() + cnt,
                                  sizeof(double) * 2 * cnt, sizeof(double) * cnt, S, cudaMemcpyDeviceToDevice, s));
      }
    } else {
      gram<double>(s, S, S - Sold, static_cast<int>(ov), w.V.get(), static_cast<int>(ov), w.S1.get() + Sold * ov,
                   static_cast<int>(ov), w.a1.get() + Sold, Smax, 1.0, 0.0, w.gws);
      if (rpa)
        gram<double>(s, S, S - Sold, static_cast<int>(ov), w.V.get(), static_cast<int>(ov), w.S2.get() + Sold * ov,
                     static_cast<int>(ov), w.a2.get() + Sold, Smax, 1.0, 0.0, w.gws);
    }
    const int k = std::min(kk, S);
    if (!rpa) {
      sym_upper(s, S, w.a1.get(), Smax, w.E.get(), S);
      kq = std::min(S, 2 * kk);
      syevk(s, S, kq, w.E.get(), S, w.w.get(), w.Q.get(), kq, w.eig_ws, w.flag.get());
      XS_CUDA(cudaMemcpyAsync(w.omega.get(), w.w.get(), sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
      // Ritz vectors and residuals
      if (w.oz) {
        // X (rows 0..kk-1 of w.X) and R = A X - omega X (rows kk.., i.e. w.AX) in one pass
        cis_coef_kernel<<<grid1((long long)S * 2 * kk, 256), 256, 0, s>>>(S, k, kk, w.Q.get(), kq, w.omega.get(),
                                                                          w.coef.get());
        XS_CHECK_LAUNCH();
        const OzBlock blk[2] = {{w.S1nn.get(), w.ldk, w.eS1.get(), w.coef.get(), 2 * kk},
                                {w.Vnn.get(), w.ldk, w.eV.get(), w.coef.get() + (size_t)S * 2 * kk, 2 * kk}};
        oz_combine(s, 2, blk, S, 2 * kk, ov, 1.0, 0.0, w.X.get(), ov, w.ozw, c.tc_err.get());
        R1p = w.AX;
        row_norms(s, k, ov, R1p, w.nrm.get());
      } else {
        gemm<double>(s, true, false, k, static_cast<int>(ov), S, 1.0, w.Q.get(), kq, 0, w.V.get(),
                     static_cast<int>(ov), 0, 0.0, w.X.get(), static_cast<int>(ov), 0, 1);
        gemm<double>(s, true, false, k, static_cast<int>(ov), S, 1.0, w.Q.get(), kq, 0, w.S1.get(),
                     static_cast<int>(ov), 0, 0.0, w.AX, static_cast<int>(ov), 0, 1);
        residual_norms(s, k, ov, w.AX, w.X.get(), w.omega.get(), w.nrm.get(), R1p);
      }
      const auto st_words = fetch(k, k);
      if (st_words.second) check_device_error(c);
    } else {
      // a- = L L^T (Cholesky; failure = unstable reference), M = L^T a+ L
      XS_CUDA(cudaMemsetAsync(w.flag.get() + 3, 0, sizeof(int), s));
      sym_upper(s, S, w.a2.get(), Smax, w.Sh.get(), S);   // Sh <- a-, factored in place into L
      // a non-positive pivot (unstable reference) is read back with the
      // residual norms below; the launches in between run on whatever the
      // factor holds and their results are discarded
      cholesky(s, S, w.Sh.get(), S, w.flag.get() + 3);
      sym_upper(s, S, w.a1.get(), Smax, w.E2.get(), S);   // E2 = a+
      gemm<double>(s, true, false, S, S, S, 1.0, w.Sh.get(), S, 0, w.E2.get(), S, 0, 0.0, w.tS.get(), S, 0, 1);
      gemm<double>(s, false, false, S, S, S, 1.0, w.tS.get(), S, 0, w.Sh.get(), S, 0, 0.0, w.E.get(), S, 0, 1);
      syevk(s, S, k, w.E.get(), S, w.w.get(), w.Q.get(), k, w.eig_ws, w.flag.get());
      sqrt_roots(s, k, w.w.get(), w.omega.get(), w.flag.get() + 3);
      // u~ = L z / sqrt(omega) (S x k), w~ = a+ u~ / omega
      gemm<double>(s, false, false, S, k, S, 1.0, w.Sh.get(), S, 0, w.Q.get(), k, 0, 0.0, w.cu.get(), k, 0, 1);
      scale_cols(s, S, k, w.cu.get(), k, w.omega.get(), 1);
      gemm<double>(s, false, false, S, k, S, 1.0, w.E2.get(), S, 0, w.cu.get(), k, 0, 0.0, w.cw.get(), k, 0, 1);
      scale_cols(s, S, k, w.cw.get(), k, w.omega.get(), 2);
      if (w.oz) {
        // residuals r1, r2 over ((A+B) V, V, (A-B) V) in one pass, then
        // [X+Y; X-Y] = [u~ w~]^T V (X+Y in X, X-Y in AX = X + kk ov)
        rpa_coef_kernel<<<grid1((long long)S * 2 * kk, 256), 256, 0, s>>>(S, k, kk, w.cu.get(), w.cw.get(),
                                                                          w.omega.get(), w.coef.get());
        XS_CHECK_LAUNCH();
        const size_t cb = (size_t)S * 2 * kk;
        const OzBlock blk[3] = {{w.S1nn.get(), w.ldk, w.eS1.get(), w.coef.get(), 2 * kk},
                                {w.Vnn.get(), w.ldk, w.eV.get(), w.coef.get() + cb, 2 * kk},
                                {w.S2nn.get(), w.ldk, w.eS2.get(), w.coef.get() + 2 * cb, 2 * kk}};
        oz_combine(s, 3, blk, S, 2 * kk, ov, 1.0, 0.0, R1p, ov, w.ozw, c.tc_err.get());
        XS_CUDA(cudaMemcpyAsync(w.rcoef.get(), w.coef.get() + 3 * cb, sizeof(double) * cb, cudaMemcpyDeviceToDevice,
                                s));
        ritz_pending = true;
        ritz_S = S;
        row_norms(s, k, ov, R1p, w.nrm.get());
        row_norms(s, k, ov, R2p, w.nrm.get() + kk);
      } else {
      // [X+Y; X-Y] = [u~ w~]^T V in one product (X+Y in X, X-Y in AX = X + kk ov),
      // then (A+B)(X+Y) (R1 scratch) and (A-B)(X-Y) (MW)
      if (k == kk) {
        XS_CUDA(cudaMemcpy2DAsync(w.tS.get(), sizeof(double) * 2 * k, w.cu.get(), sizeof(double) * k,
                                  sizeof(double) * k, S, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpy2DAsync(w.tS.get() + k, sizeof(double) * 2 * k, w.cw.get(), sizeof(double) * k,
                                  sizeof(double) * k, S, cudaMemcpyDeviceToDevice, s));
        gemm<double>(s, true, false, 2 * k, static_cast<int>(ov), S, 1.0, w.tS.get(), 2 * k, 0, w.V.get(),
                     static_cast<int>(ov), 0, 0.0, w.X.get(), static_cast<int>(ov), 0, 1);
      } else {
        gemm<double>(s, true, false, k, static_cast<int>(ov), S, 1.0, w.cu.get(), k, 0, w.V.get(),
                     static_cast<int>(ov), 0, 0.0, w.X.get(), static_cast<int>(ov), 0, 1);
        gemm<double>(s, true, false, k, static_cast<int>(ov), S, 1.0, w.cw.get(), k, 0, w.V.get(),
                     static_cast<int>(ov), 0, 0.0, w.AX, static_cast<int>(ov), 0, 1);
      }
      gemm<double>(s, true, false, k, static_cast<int>(ov), S, 1.0, w.cu.get(), k, 0, w.S1.get(), static_cast<int>(ov),
                   0, 0.0, R1p, static_cast<int>(ov), 0, 1);
      gemm<double>(s, true, false, k, static_cast<int>(ov), S, 1.0, w.cw.get(), k, 0, w.S2.get(), static_cast<int>(ov),
                   0, 0.0, w.MW.get(), static_cast<int>(ov), 0, 1);
      // r1 = (A+B)(X+Y) - omega (X-Y), r2 = (A-B)(X-Y) - omega (X+Y)
      residual_norms(s, k, ov, R1p, w.AX, w.omega.get(), w.nrm.get(), R1p);
      residual_norms(s, k, ov, w.MW.get(), w.X.get(), w.omega.get(), w.nrm.get() + kk, R2p);
      }
      const auto st_words = fetch(k, 2 * kk);
      if (st_words.first) {
        // unstable reference: later launches saw a garbage factor; drop their error word
        if (c.tc_err.get()) XS_CUDA(cudaMemsetAsync(c.tc_err.get(), 0, sizeof(int), s));
        status = XS_EUNSTABLE;
        break;
      }
      if (st_words.second) check_device_error(c);
      for (int j = 0; j < k; ++j) hn[j] = std::max(hn[j], hn[kk + j]);
    }
    bool all = true;
    for (int j = 0; j < k; ++j) {
      if (!std::isfinite(hn[j]) || !std::isfinite(hw[j])) throw Error(XS_ECUDA, "non-finite Davidson residual");
      conv[j] = hn[j] <= tol_eff;
      all = all && conv[j];
    }
    if (polishing) { converged = true; st.polished = true; break; }
    if ((all && k == kk) || it >= max_iter) flush_ritz();
    if (all && k == kk) {
      if (opt.precision == XS_MIXED) {
        // Rayleigh-Ritz once more in the span of the converged Ritz vectors
        // with float32 SIMT products: the tensor cores' float32 accumulation
        // truncates, which biases their products by ~1e-5 relative; the
        // round-to-nearest SIMT products remove that bias from the energies.
        const int nrows = rpa ? 2 * k : k;
        XS_CUDA(cudaMemcpyAsync(w.T.get(), w.X.get(), sizeof(double) * k * ov, cudaMemcpyDeviceToDevice, s));
        if (rpa)
          XS_CUDA(cudaMemcpyAsync(w.T.get() + (size_t)k * ov, w.AX, sizeof(double) * k * ov,
                                  cudaMemcpyDeviceToDevice, s));
        const int nb = orthonormalise_append(c, w, 0, nrows, ov, w.V.get(), w.oz ? w.mxV.get() : nullptr);
        if (nb >= k) {
          slice_V(c, w, ov, 0, nb, w.oz ? w.mxV.get() : nullptr);
          prod_prec = kPrecF32;
          apply(0, nb);
          S = nb;
          Sold = 0;
          polishing = true;
          continue;
        }
      }
      converged = true;
      break;
    }
    if (it >= max_iter) break;
    // preconditioned residuals of the unconverged roots
    // fallback: drop the learned shift when the largest residual has not
    // fallen by 10% over the last five iterations
    max_res_hist.push_back(*std::max_element(hn.begin(), hn.begin() + k));
    if (shift && max_res_hist.size() > 5 &&
        max_res_hist.back() > 0.9 * max_res_hist[max_res_hist.size() - 6]) {
      shift = nullptr;
      st.fallback = true;
    }
    precondition(s, k, o, v, m.eps.get(), w.omega.get(), R1p, R1p, shift);
    if (rpa) precondition(s, k, o, v, m.eps.get(), w.omega.get(), R2p, R2p, shift);
    // new directions, roots with the largest residual first.  When the
    // subspace has room for only part of the block but for at least a quarter
    // of it, the part that fits is appended and the restart waits; below
    // that, V is collapsed onto the current Ritz vectors first.
    std::vector<int> order;
    for (int j = 0; j < k; ++j)
      if (!conv[j]) order.push_back(j);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hn[x] > hn[y]; });
    const int per = rpa ? 2 : 1;
    const int want = static_cast<int>(order.size()) * per;
    const bool restart = want > Smax - S && Smax - S < std::max(per, want / 4);
    const int take = (restart || want <= Smax - S) ? static_cast<int>(order.size()) : (Smax - S) / per;
    int nnew = 0;
    for (int q = 0; q < take; ++q) {
      const int j = order[q];
      XS_CUDA(cudaMemcpyAsync(w.T.get() + nnew * ov, R1p + j * ov, sizeof(double) * ov,
                              cudaMemcpyDeviceToDevice, s));
      ++nnew;
      if (rpa) {
        XS_CUDA(cudaMemcpyAsync(w.T.get() + nnew * ov, R2p + j * ov, sizeof(double) * ov,
                                cudaMemcpyDeviceToDevice, s));
        ++nnew;
      }
    }
    if (restart) {
      // collapse onto the current Ritz vectors (which the deferred Ritz
      // combination needs in the old basis)
      flush_ritz();
      int nc;
      if (!rpa) {
        nc = kq;
        w.C1.ensure((size_t)nc * ov);
        w.C2.ensure((size_t)nc * ov);
        if (w.oz) {
          const OzBlock bv{w.Vnn.get(), w.ldk, w.eV.get(), w.Q.get(), kq};
          const OzBlock bs{w.S1nn.get(), w.ldk, w.eS1.get(), w.Q.get(), kq};
          oz_combine(s, 1, &bv, S, nc, ov, 1.0, 0.0, w.C1.get(), ov, w.ozw, c.tc_err.get());
          oz_combine(s, 1, &bs, S, nc, ov, 1.0, 0.0, w.C2.get(), ov, w.ozw, c.tc_err.get());
        } else {
          gemm<double>(s, true, false, nc, static_cast<int>(ov), S, 1.0, w.Q.get(), kq, 0, w.V.get(),
                       static_cast<int>(ov), 0, 0.0, w.C1.get(), static_cast<int>(ov), 0, 1);
          gemm<double>(s, true, false, nc, static_cast<int>(ov), S, 1.0, w.Q.get(), kq, 0, w.S1.get(),
                       static_cast<int>(ov), 0, 0.0, w.C2.get(), static_cast<int>(ov), 0, 1);
        }
        XS_CUDA(cudaMemcpyAsync(w.V.get(), w.C1.get(), sizeof(double) * nc * ov, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpyAsync(w.S1.get(), w.C2.get(), sizeof(double) * nc * ov, cudaMemcpyDeviceToDevice, s));
        set_diag(s, nc, w.w.get(), w.a1.get(), Smax);
        slice_V(c, w, ov, 0, nc);
        slice_P(c, w, ov, w.S1.get(), w.eS1, w.S1nn, 0, nc, false);
      } else {
        // orthonormal basis of span{u~, w~} in subspace coordinates
        XS_CUDA(cudaMemcpy2DAsync(w.tS.get(), sizeof(double) * 2 * k, w.cu.get(), sizeof(double) * k,
                                  sizeof(double) * k, S, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpy2DAsync(w.tS.get() + k, sizeof(double) * 2 * k, w.cw.get(), sizeof(double) * k,
                                  sizeof(double) * k, S, cudaMemcpyDeviceToDevice, s));
        // Gram (2k x 2k) of the coefficient columns
        gemm<double>(s, true, false, 2 * k, 2 * k, S, 1.0, w.tS.get(), 2 * k, 0, w.tS.get(), 2 * k, 0, 0.0,
                     w.E2.get(), 2 * k, 0, 1);
        jacobi_eig(s, 2 * k, w.E2.get(), 2 * k, w.Q2.get(), 2 * k, w.w2.get(), w.flag.get() + 1);
        lowdin(s, 2 * k, w.w2.get(), w.Q2.get(), 2 * k, kLowdinThresh, w.Bm.get(), 2 * k, w.flag.get() + 2);
        sync_copy(s, &nc, w.flag.get() + 2, sizeof(int));
        // Cn = Ycoef Bm^T (S x nc)
        gemm<double>(s, false, true, S, nc, 2 * k, 1.0, w.tS.get(), 2 * k, 0, w.Bm.get(), 2 * k, 0, 0.0, w.E.get(),
                     nc, 0, 1);
        w.C1.ensure((size_t)nc * ov);
        w.C2.ensure((size_t)nc * ov);
        w.C3.ensure((size_t)nc * ov);
        if (w.oz) {
          const OzBlock b1{w.Vnn.get(), w.ldk, w.eV.get(), w.E.get(), nc};
          const OzBlock b2{w.S1nn.get(), w.ldk, w.eS1.get(), w.E.get(), nc};
          const OzBlock b3{w.S2nn.get(), w.ldk, w.eS2.get(), w.E.get(), nc};
          oz_combine(s, 1, &b1, S, nc, ov, 1.0, 0.0, w.C1.get(), ov, w.ozw, c.tc_err.get());
          oz_combine(s, 1, &b2, S, nc, ov, 1.0, 0.0, w.C2.get(), ov, w.ozw, c.tc_err.get());
          oz_combine(s, 1, &b3, S, nc, ov, 1.0, 0.0, w.C3.get(), ov, w.ozw, c.tc_err.get());
        } else {
          gemm<double>(s, true, false, nc, static_cast<int>(ov), S, 1.0, w.E.get(), nc, 0, w.V.get(),
                       static_cast<int>(ov), 0, 0.0, w.C1.get(), static_cast<int>(ov), 0, 1);
          gemm<double>(s, true, false, nc, static_cast<int>(ov), S, 1.0, w.E.get(), nc, 0, w.S1.get(),
                       static_cast<int>(ov), 0, 0.0, w.C2.get(), static_cast<int>(ov), 0, 1);
          gemm<double>(s, true, false, nc, static_cast<int>(ov), S, 1.0, w.E.get(), nc, 0, w.S2.get(),
                       static_cast<int>(ov), 0, 0.0, w.C3.get(), static_cast<int>(ov), 0, 1);
        }
        XS_CUDA(cudaMemcpyAsync(w.V.get(), w.C1.get(), sizeof(double) * nc * ov, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpyAsync(w.S1.get(), w.C2.get(), sizeof(double) * nc * ov, cudaMemcpyDeviceToDevice, s));
        XS_CUDA(cudaMemcpyAsync(w.S2.get(), w.C3.get(), sizeof(double) * nc * ov, cudaMemcpyDeviceToDevice, s));
        if (w.oz) {
          slice_V(c, w, ov, 0, nc);
          slice_P(c, w, ov, w.S1.get(), w.eS1, w.S1nn, 0, nc, true);
          oz_gram(s, nc, nc, ov, w.Vtn.get(), w.Pv, w.eV.get(), w.Btn.get(), w.Pb, w.eS1.get(), 1.0, 0.0,
                  w.a1.get(), Smax, w.ozw, c.tc_err.get());
          slice_P(c, w, ov, w.S2.get(), w.eS2, w.S2nn, 0, nc, true);
          oz_gram(s, nc, nc, ov, w.Vtn.get(), w.Pv, w.eV.get(), w.Btn.get(), w.Pb, w.eS2.get(), 1.0, 0.0,
                  w.a2.get(), Smax, w.ozw, c.tc_err.get());
        } else {
          gram<double>(s, nc, nc, static_cast<int>(ov), w.V.get(), static_cast<int>(ov), w.S1.get(),
                       static_cast<int>(ov), w.a1.get(), Smax, 1.0, 0.0, w.gws);
          gram<double>(s, nc, nc, static_cast<int>(ov), w.V.get(), static_cast<int>(ov), w.S2.get(),
                       static_cast<int>(ov), w.a2.get(), Smax, 1.0, 0.0, w.gws);
        }
      }
      S = nc;
      st.collapses += 1;
    }
    nnew = std::min(nnew, Smax - S);
    if (nnew <= 0) break;  // the subspace already spans everything it can hold
    int nkeep = orthonormalise_append(c, w, S, nnew, ov, w.V.get() + (size_t)S * ov,
                                      w.oz ? w.mxV.get() + S : nullptr);
    if (nkeep == 0) break;  // no new direction: stagnation
    slice_V(c, w, ov, S, nkeep, w.oz ? w.mxV.get() + S : nullptr);
    Sold = S;
    S += nkeep;
    apply(Sold, nkeep);
  }
  h_loop.stop();
  HostScope h_finish("host:finish");
  if (status == XS_OK) flush_ritz();   // V rows < ritz_S are unchanged since the last Rayleigh-Ritz step
  check_device_error(c);
  st.iterations = std::min(it, max_iter);
  {
    XS_CUDA(cudaStreamSynchronize(s));
    double ms_total = 0.0;
    for (auto& e : prod_events) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) ms_total += ms;
    }
    st.seconds_products = ms_total / 1e3;
  }
  if (status != XS_OK) return status;

  // keep the roots: U = X+Y (CIS: X), W = X-Y (CIS: X)
  m.nroots = kk;
  m.method = opt.method;
  m.spin = opt.spin;
  m.U.alloc((size_t)kk * ov);
  m.Wv.alloc((size_t)kk * ov);
  XS_CUDA(cudaMemcpyAsync(m.U.get(), w.X.get(), sizeof(double) * kk * ov, cudaMemcpyDeviceToDevice, s));
  XS_CUDA(cudaMemcpyAsync(m.Wv.get(), rpa ? w.AX : w.X.get(), sizeof(double) * kk * ov,
                          cudaMemcpyDeviceToDevice, s));
  m.omega.assign(hw.begin(), hw.begin() + kk);
  m.resid.assign(hn.begin(), hn.begin() + kk);
  m.osc.assign(kk, 0.0);   // triplets: dipole-forbidden
  if (!triplet) {
    w.fdev.ensure(kk);
    oscillator_strengths(c, m, kk, m.U.get(), w.omega.get(), w.fdev.get());
    sync_copy(s, m.osc.data(), w.fdev.get(), sizeof(double) * kk);
  }
  m.iterations = st.iterations;
  st.converged = converged;
  return converged ? XS_OK : XS_ENOCONV;
}

}  // namespace xs
