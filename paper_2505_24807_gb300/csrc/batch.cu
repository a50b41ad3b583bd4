// Lock-step batched Davidson of libxs (paper, Section "GPU Implementation",
// batched steps 1-6; the batch mode of Section "Results and discussion").
//
// All molecules of one xs_ground_state call are solved together.  Each keeps
// its own subspace (no zero padding, no padding roots to discard), and the
// whole batch advances one Davidson iteration per replay of one captured CUDA
// graph.  The graph is a fixed sequence of ragged kernels: every kernel reads
// the per-molecule counts (vectors to multiply, subspace size, new directions,
// status) from device memory, forms its work list over all molecules in its
// prologue (a prefix sum of per-molecule work units in shared memory) and
// walks it with a persistent grid.  A molecule whose roots have converged
// contributes no work units from then on: it retires on the device while the
// rest continue.  The host replays the graph and reads one word per iteration
// (the number of molecules still active).
//
// One iteration:
//   products of the vectors appended in the previous iteration (step 2):
//     P1  T_j = C_occ X_j                                     (per vector)
//     P2  R = [T_1; T_2; ..] C_vir^T                          (vectors stacked)
//     G   diagonal blocks packed, J2 = W r, atom-pair tiles of G (and G-)
//     B1  S = [G_1; G_2; ..] C_vir                            (stacked; G+ and G-)
//     B2  (A V)_j = C_occ^T S_j + (eps_a - eps_i) X_j         (per vector, float64)
//   (the n^2 contractions run over nvir, never larger than nocc for neutral
//   H/C/N/O molecules); products in float32 (XS_MIXED: float32 SIMT with
//   round-to-nearest accumulation) or float64 (XS_FP64);
//   float64 subspace (steps 3-6): new columns of the projected matrices, the
//   lowest eigenpairs (one CTA per molecule; TDHF in the symmetric form of
//   Stratmann, Scuseria and Frisch), Ritz vectors and residuals, their norms,
//   convergence and restart decisions, preconditioned residuals, collapse onto
//   the Ritz vectors when the subspace is full, two classical Gram-Schmidt
//   passes, Loewdin orthonormalisation of the new block, append.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "batch.h"
#include "gbuild_dev.cuh"
#include "gpair_dev.cuh"
#include "jacobi.cuh"
#include "kernels.h"
#include "mlp.h"
#include "syev_body.cuh"

namespace xs {

namespace {

// ---- per-molecule state (int words on the device) --------------------------
enum StField {
  F_S = 0,      // stored vectors
  F_SOLD,       // first vector of the last appended block
  F_NNEW,       // vectors to multiply in this iteration's products
  F_STATUS,     // BS_*
  F_ITER,       // Rayleigh-Ritz steps taken
  F_NDIR,       // new directions in T
  F_COLL,       // 1: collapse this iteration
  F_NC,         // subspace size after the collapse
  F_NKEEP,      // directions kept by the Loewdin step
  F_KQ,         // eigenvectors kept by the eigensolver (CIS)
  F_PROD,       // trial vectors multiplied so far
  F_GS2,        // 1: a second Gram-Schmidt pass is needed
  F_NOSHIFT,    // 1: the learned shift was dropped (a residual stalled)
  kSt = 16
};
enum Status { BS_ACTIVE = 0, BS_CONVERGED = 1, BS_STALLED = 2, BS_MAXITER = 3, BS_UNSTABLE = 4 };

constexpr double kLowdinThresh = 1e-14;
constexpr double kMixedResidualFloor = 1e-4;
constexpr int kGramChunk = 1024;   // amplitudes per partial Gram block
constexpr int kCombChunk = 256;    // amplitudes per combination work unit

// ---- per-molecule descriptor (device) ----------------------------------------
struct BMol {
  int n, o, v, np, natoms;
  long long ov;
  int kk, maxnew, pmax, Smax, nch;
  int ntr, ntc;                       // G tiles: row groups, column tiles
  const int4* gb_rows;
  const int4* gb_cols;
  const int2* gp_pairs;               // super-atom pairs of the float32 G build
  const int4* gp_sa;
  int gp_npairs;
  const int *ao_atom, *ao_local, *atom_ao_off, *atom_nao, *atom_prod_off, *atom_elem;
  const double* eps;
  const double* dip;                  // MO dipole integrals 3 x ov
  const void* CT;                     // MO-major coefficients (product type)
  const void* W;                      // two-centre supermatrix (product type)
  // float64 subspace
  double *V, *S1, *S2;                // Smax x ov
  double *Xb, *Rb, *T, *C;            // Ritz rows (2kk), TDHF residual rows (2kk), new directions, collapse
  double *a1, *a2, *Q, *E, *coef, *tS, *G2, *Bm, *Mb, *Lb, *Pb, *Nb;   // small matrices
  double *wts, *omega, *nrm, *tn, *dm, *osc, *gpart, *syw;
  int* slot;                          // new direction -> root * 2 + residual kind
  double *U, *Wv;                     // the molecule's kept amplitudes (X+Y and X-Y; CIS: X and X)
  double* shift;                      // learned diagonal shift (ov) or null
  double* rhist;                      // largest residual of the last 8 iterations
  // product scratch (product type)
  void *Xf, *Tm, *Rm, *Gp, *Gq, *Sb, *Sq, *r, *J2;
};

struct BCfg {
  int nmol;
  int rpa, triplet, coulomb, mode;    // GMode of the G build
  int max_iter;
  double tol;
  int pass;                           // Gram-Schmidt pass of the launch (0 or 1)
  int smax;                           // largest subspace cap of the group
};

__device__ __forceinline__ double de_of(const BMol& d, long long l) {
  const int i = static_cast<int>(l / d.v), a = static_cast<int>(l - (long long)i * d.v);
  return d.eps[d.o + a] - d.eps[i];
}

// Exclusive prefix of per-molecule work units in shared memory (pref[0..nmol]),
// computed by the whole CTA; returns the total.  units(m) must be the same in
// every CTA of a launch (it reads state that no kernel of the launch writes).
template <typename F>
__device__ int block_prefix(int nmol, F units, int* pref) {
  __shared__ int wsum[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (nmol + nt - 1) / nt;
  const int m0 = tid * per, m1 = min(nmol, m0 + per);
  int loc = 0;
  for (int m = m0; m < m1; ++m) loc += units(m);
  // inclusive scan of loc over the CTA
  const int lane = tid & 31, w = tid >> 5;
  int x = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = nt >> 5;
    int s = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) wsum[lane] = s;
  }
  __syncthreads();
  int run = x - loc + (w > 0 ? wsum[w - 1] : 0);
  for (int m = m0; m < m1; ++m) {
    pref[m] = run;
    run += units(m);
  }
  if (tid == nt - 1) pref[nmol] = run;
  __syncthreads();
  return pref[nmol];
}

// molecule owning work unit u: the largest m with pref[m] <= u
__device__ __forceinline__ int find_mol(const int* pref, int nmol, int u) {
  int lo = 0, hi = nmol - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool active(const int* st, int m) { return st[m * kSt + F_STATUS] == BS_ACTIVE; }
__device__ __forceinline__ int sf(const int* st, int m, int f) { return st[m * kSt + f]; }

#define RAGGED_PROLOGUE(UNITS)                                   \
  __shared__ int pref[kBatchGroup + 1];                          \
  const int total = block_prefix(cfg.nmol, UNITS, pref);         \
  for (int u = blockIdx.x; u < total; u += gridDim.x)

__host__ __device__ __forceinline__ int cdiv(long long a, int b) { return static_cast<int>((a + b - 1) / b); }

// ---- ragged SIMT GEMM of the products ---------------------------------------
// 64 x 64 output tiles, K blocks of 16, 256 threads with 4 x 4 outputs each,
// round-to-nearest accumulation in the product type.
enum GRole { R_P1 = 0, R_P2, R_J2, R_B1, R_B2 };
constexpr int kBM = 64, kBN = 64, kBK = 16;

template <typename T>
struct GP {
  const T* A;
  const T* B;
  T* C;
  double* Cd;         // float64 output with the orbital-energy term (R_B2)
  const double* X;    // its trial vector
  int M, N, K, lda, ldb, ldc;
};

template <int ROLE>
__device__ __forceinline__ int gemm_units(const BMol& d, const int* st, int m, const BCfg& cfg) {
  if (!active(st, m)) return 0;
  const int cnt = sf(st, m, F_NNEW);
  if (cnt <= 0) return 0;
  const int nw = cfg.rpa ? 2 : 1;
  switch (ROLE) {
    case R_P1: return cdiv(d.n, kBM) * cdiv(d.v, kBN) * cnt;
    case R_P2: return cdiv((long long)cnt * d.n, kBM) * cdiv(d.n, kBN);
    case R_J2: return cfg.coulomb ? cdiv(d.np, kBM) * cdiv(cnt, kBN) : 0;
    case R_B1: return cdiv((long long)cnt * d.n, kBM) * cdiv(d.v, kBN) * nw;
    default: return cdiv(d.o, kBM) * cdiv(d.v, kBN) * cnt * nw;
  }
}

// the problem of work unit lu of molecule d, and its output tile origin
template <typename T, int ROLE>
__device__ __forceinline__ GP<T> gemm_problem(const BMol& d, const int* st, int m, int lu, int& m0, int& n0) {
  const int cnt = sf(st, m, F_NNEW), sold = sf(st, m, F_SOLD);
  const T* CT = static_cast<const T*>(d.CT);
  const T* CTvir = CT + (size_t)d.o * d.n;
  GP<T> p{};
  int tm = 0, tn = 0;
  switch (ROLE) {
    case R_P1: tm = cdiv(d.n, kBM); tn = cdiv(d.v, kBN); break;
    case R_P2: tm = cdiv((long long)cnt * d.n, kBM); tn = cdiv(d.n, kBN); break;
    case R_J2: tm = cdiv(d.np, kBM); tn = cdiv(cnt, kBN); break;
    case R_B1: tm = cdiv((long long)cnt * d.n, kBM); tn = cdiv(d.v, kBN); break;
    default: tm = cdiv(d.o, kBM); tn = cdiv(d.v, kBN); break;
  }
  const int b = lu / (tm * tn), t = lu - b * (tm * tn);
  m0 = (t / tn) * kBM;
  n0 = (t % tn) * kBN;
  if (ROLE == R_P1) {   // T_j (n x v) = C_occ X_j: A = CT rows 0..o-1 read transposed
    p.A = CT; p.lda = d.n;
    if (sizeof(T) == 4) p.B = static_cast<const T*>(d.Xf) + (size_t)b * d.ov;
    else p.B = reinterpret_cast<const T*>(d.V + (size_t)(sold + b) * d.ov);
    p.ldb = d.v;
    p.C = static_cast<T*>(d.Tm) + (size_t)b * d.n * d.v; p.ldc = d.v;
    p.M = d.n; p.N = d.v; p.K = d.o;
  } else if (ROLE == R_P2) {   // R = [T_j] C_vir^T
    p.A = static_cast<const T*>(d.Tm); p.lda = d.v;
    p.B = CTvir; p.ldb = d.n;
    p.C = static_cast<T*>(d.Rm); p.ldc = d.n;
    p.M = cnt * d.n; p.N = d.n; p.K = d.v;
  } else if (ROLE == R_J2) {   // J2 = W r
    p.A = static_cast<const T*>(d.W); p.lda = d.np;
    p.B = static_cast<const T*>(d.r); p.ldb = d.pmax;
    p.C = static_cast<T*>(d.J2); p.ldc = d.pmax;
    p.M = d.np; p.N = cnt; p.K = d.np;
  } else if (ROLE == R_B1) {   // S = [G_j] C_vir: B = CT rows o.. read transposed
    p.A = static_cast<const T*>(b ? d.Gq : d.Gp); p.lda = d.n;
    p.B = CTvir; p.ldb = d.n;
    p.C = static_cast<T*>(b ? d.Sq : d.Sb); p.ldc = d.v;
    p.M = cnt * d.n; p.N = d.v; p.K = d.n;
  } else {   // (A V)_j = C_occ^T S_j + de X_j
    const int which = b / cnt, j = b - which * cnt;
    p.A = CT; p.lda = d.n;
    p.B = static_cast<const T*>(which ? d.Sq : d.Sb) + (size_t)j * d.n * d.v; p.ldb = d.v;
    p.Cd = (which ? d.S2 : d.S1) + (size_t)(sold + j) * d.ov; p.ldc = d.v;
    p.X = d.V + (size_t)(sold + j) * d.ov;
    p.M = d.o; p.N = d.v; p.K = d.n;
  }
  return p;
}

template <typename T, int ROLE>
__global__ void __launch_bounds__(256) bgemm_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  constexpr bool TA = ROLE == R_P1, TB = ROLE == R_B1;
  __shared__ __align__(16) T As[kBK][kBM + 4];
  __shared__ __align__(16) T Bs[kBK][kBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  RAGGED_PROLOGUE([&](int m) { return gemm_units<ROLE>(mols[m], st, m, cfg); }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    int m0, n0;
    const GP<T> p = gemm_problem<T, ROLE>(d, st, m, u - pref[m], m0, n0);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < p.K; k0 += kBK) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q;
        // A tile (op(A) rows m0.., columns k0..) into As[k][m]
        if (TA) {
          const int kk = e / kBM, mm = e % kBM;
          const int gk = k0 + kk, gm = m0 + mm;
          As[kk][mm] = (gk < p.K && gm < p.M) ? p.A[(size_t)gk * p.lda + gm] : T(0);
        } else {
          const int mm = e / kBK, kk = e % kBK;
          const int gk = k0 + kk, gm = m0 + mm;
          As[kk][mm] = (gk < p.K && gm < p.M) ? p.A[(size_t)gm * p.lda + gk] : T(0);
        }
        // B tile (op(B) rows k0.., columns n0..) into Bs[k][n]
        if (TB) {
          const int nn = e / kBK, kk = e % kBK;
          const int gk = k0 + kk, gn = n0 + nn;
          Bs[kk][nn] = (gk < p.K && gn < p.N) ? p.B[(size_t)gn * p.ldb + gk] : T(0);
        } else {
          const int kk = e / kBN, nn = e % kBN;
          const int gk = k0 + kk, gn = n0 + nn;
          Bs[kk][nn] = (gk < p.K && gn < p.N) ? p.B[(size_t)gk * p.ldb + gn] : T(0);
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kBK; ++kk) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a[i] = As[kk][ty * 4 + i];
          b[i] = Bs[kk][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty * 4 + i;
      if (gm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx * 4 + j;
        if (gn >= p.N) continue;
        if (ROLE == R_B2) {
          const size_t l = (size_t)gm * p.ldc + gn;   // amplitude (i, a)
          const double de = d.eps[d.o + gn] - d.eps[gm];
          p.Cd[l] = static_cast<double>(acc[i][j]) + de * p.X[l];
        } else {
          p.C[(size_t)gm * p.ldc + gn] = acc[i][j];
        }
      }
    }
  }
}

// X_f = float32 copy of the vectors to multiply (float32 products only)
__global__ void __launch_bounds__(256) bconvert_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                       BCfg cfg) {
  RAGGED_PROLOGUE([&](int m) {
    return active(st, m) ? sf(st, m, F_NNEW) * cdiv(mols[m].ov, 4096) : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int lu = u - pref[m], nchk = cdiv(d.ov, 4096);
    const int j = lu / nchk, c = lu - j * nchk;
    const double* src = d.V + (size_t)(sf(st, m, F_SOLD) + j) * d.ov;
    float* dst = static_cast<float*>(d.Xf) + (size_t)j * d.ov;
    const long long l0 = (long long)c * 4096, l1 = min(d.ov, l0 + 4096);
    for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) dst[l] = static_cast<float>(src[l]);
  }
}

// ---- G build of the batch ------------------------------------------------------
// product vectors of the diagonal atom blocks: r[q][j] (row stride pmax)
template <typename T>
__global__ void __launch_bounds__(256) bpack_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  RAGGED_PROLOGUE([&](int m) { return (cfg.coulomb && active(st, m)) ? sf(st, m, F_NNEW) : 0; }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int j = u - pref[m], n = d.n;
    const T* R = static_cast<const T*>(d.Rm) + (size_t)j * n * n;
    T* r = static_cast<T*>(d.r);
    for (int A = threadIdx.x; A < d.natoms; A += blockDim.x) {
      const int o = d.atom_ao_off[A], P = d.atom_prod_off[A];
      if (d.atom_nao[A] == 1) {
        r[(size_t)P * d.pmax + j] = R[(size_t)o * n + o];
      } else {
        for (int a = 0; a < 4; ++a)
          for (int b = a; b < 4; ++b) {
            T val = R[(size_t)(o + a) * n + o + b];
            if (b != a) val += R[(size_t)(o + b) * n + o + a];
            r[(size_t)(P + pidx(a, b)) * d.pmax + j] = val;
          }
      }
    }
  }
}

// Atom-aligned tiles of G for every molecule of the batch: a work unit is one
// row group (a heavy atom's 4 AOs or up to 4 hydrogens) x one column tile
// (whole atoms, at most 64 AOs) of one molecule.  The tile's pair-integral
// block is staged in shared memory once per unit; the molecule's new R
// matrices pass through the tile one by one (and, for TDHF, the transposed
// tile: K(R^T)).  The same contraction as the single-molecule G build.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) bgtile_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                     BCfg cfg, const double* __restrict__ par) {
  constexpr bool kRpa = MODE == G_RPA || MODE == G_RPA_T;
  constexpr bool kTriplet = MODE == G_CIS_T || MODE == G_RPA_T;
  __shared__ T Ws[kGP][kGQ + 1];
  __shared__ T Rt[kGR + 4][kGC + 4];
  __shared__ T Rtt[kGC + 4][kGR + 5];
  const int tid = threadIdx.x;
  RAGGED_PROLOGUE([&](int m) {
    return (active(st, m) && sf(st, m, F_NNEW) > 0) ? mols[m].ntr * mols[m].ntc : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int lu = u - pref[m];
    const int4 rg = d.gb_rows[lu / d.ntc], ct = d.gb_cols[lu % d.ntc];
    const int n = d.n, np = d.np, cnt = sf(st, m, F_NNEW);
    const T* W = static_cast<const T*>(d.W);
    const T* J2 = static_cast<const T*>(d.J2);
    const int ra = rg.x, nr = rg.y, cb = ct.x, nc = ct.y;
    const int PA0 = d.atom_prod_off[rg.z], PB0 = d.atom_prod_off[ct.z];
    const int nPA = d.atom_prod_off[rg.w - 1] + (d.atom_nao[rg.w - 1] == 4 ? 10 : 1) - PA0;
    const int nPB = d.atom_prod_off[ct.w - 1] + (d.atom_nao[ct.w - 1] == 4 ? 10 : 1) - PB0;
    __syncthreads();   // the previous unit's reads of Ws / Rt are done
    for (int pr = tid >> 5; pr < nPA; pr += blockDim.x >> 5)
      for (int pc = tid & 31; pc < nPB; pc += 32) Ws[pr][pc] = W[(size_t)(PA0 + pr) * np + PB0 + pc];
    for (int idx = tid; idx < (kGR + 4) * (kGC + 4); idx += blockDim.x) (&Rt[0][0])[idx] = T(0);
    for (int idx = tid; idx < (kGC + 4) * (kGR + 5); idx += blockDim.x) (&Rtt[0][0])[idx] = T(0);
    const int ri = tid / kGC, ci = tid % kGC;
    const bool act = ri < nr && ci < nc;
    const int mu = ra + ri, lam = cb + ci;
    int A = 0, B = 0, a = 0, b = 0, nA = 1, nB = 1, rA = 0, cA = 0, rB = 0, pA = 0, pB = 0, PA = 0;
    const double* pd = par;
    if (act) {
      A = d.ao_atom[mu]; B = d.ao_atom[lam];
      a = d.ao_local[mu]; b = d.ao_local[lam];
      nA = d.atom_nao[A]; nB = d.atom_nao[B];
      rA = d.atom_ao_off[A] - ra;
      cA = d.atom_ao_off[A] - cb;
      rB = d.atom_ao_off[B] - cb;
      PA = d.atom_prod_off[A];
      pA = PA - PA0;
      pB = d.atom_prod_off[B] - PB0;
      if (A == B) pd = par + d.atom_elem[A] * XS_NPARAM;
    }
    __syncthreads();
    T wv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) wv[q] = T(0);
    if (act && A != B) {
#pragma unroll
      for (int nu = 0; nu < 4; ++nu)
#pragma unroll
        for (int sg = 0; sg < 4; ++sg)
          if (nu < nA && sg < nB)
            wv[nu * 4 + sg] = Ws[pA + ((nA == 4) ? pidx(a, nu) : 0)][pB + ((nB == 4) ? pidx(b, sg) : 0)];
    }
    const int tr = tid % kGR, tc = tid / kGR;
    const bool tact = kRpa && tr < nr && tc < nc;
    const size_t nn = (size_t)n * n;
    const size_t at_r = (size_t)mu * n + lam, at_t = (size_t)(cb + tc) * n + ra + tr;
    const T* Rall = static_cast<const T*>(d.Rm);
    T* Gp = static_cast<T*>(d.Gp);
    T* Gq = static_cast<T*>(d.Gq);
    for (int j = 0; j < cnt; ++j) {
      __syncthreads();
      if (act) Rt[ri][ci] = Rall[j * nn + at_r];
      if (tact) Rtt[tc][tr] = Rall[j * nn + at_t];
      __syncthreads();
      if (!act) continue;
      T g, gm = T(0);
      if (A == B) {
        T J1, K1ab, K1ba;
        if (nA == 1) {
          const T r00 = Rt[rA][cA];
          const T gss = T(pd[4]);
          J1 = gss * r00;
          K1ab = K1ba = gss * r00;
        } else {
          T Rd[16];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) Rd[i * 4 + q] = Rt[rA + i][cA + q];
          T p[XS_NPARAM];
#pragma unroll
          for (int i = 0; i < XS_NPARAM; ++i) p[i] = (i >= 4 && i <= 8) ? T(pd[i]) : T(0);
          one_centre<T>(p, a, b, Rd, J1, K1ab, K1ba);
        }
        if constexpr (kTriplet) {
          (void)J1;
          g = kRpa ? -(K1ab + K1ba) : -K1ab;
          if (kRpa) gm = -(K1ab - K1ba);
        } else {
          const int pab = (nA == 4) ? pidx(a, b) : 0;
          const T J = J1 + J2[(size_t)(PA + pab) * d.pmax + j];
          if (!kRpa) {
            g = T(2) * J - K1ab;
          } else {
            g = T(4) * J - (K1ab + K1ba);
            gm = -(K1ab - K1ba);
          }
        }
      } else {
        T kr = T(0), krt = T(0);
#pragma unroll
        for (int nu = 0; nu < 4; ++nu)
#pragma unroll
          for (int sg = 0; sg < 4; ++sg) {
            kr = fma(wv[nu * 4 + sg], Rt[rA + nu][rB + sg], kr);
            if (kRpa) krt = fma(wv[nu * 4 + sg], Rtt[rB + sg][rA + nu], krt);
          }
        if (!kRpa) {
          g = -kr;
        } else {
          g = -(kr + krt);
          gm = -(kr - krt);
        }
      }
      Gp[j * nn + at_r] = g;
      if (kRpa) Gq[j * nn + at_r] = gm;
    }
  }
}

// float32 G build of the batch over each molecule's super-atom pairs (the
// single-molecule pair build, gpair.cu): a work unit is 256 pairs of one
// molecule, every pair through all of the molecule's new matrices
template <int MODE>
__global__ void __launch_bounds__(256, 2) bgpair_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                        BCfg cfg, const double* __restrict__ par) {
  extern __shared__ float wsm[];   // 100 integrals per thread
  RAGGED_PROLOGUE([&](int m) {
    return (active(st, m) && sf(st, m, F_NNEW) > 0) ? cdiv(mols[m].gp_npairs, 256) : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int t = (u - pref[m]) * 256 + threadIdx.x;
    if (t >= d.gp_npairs) continue;
    PairOut o{static_cast<float*>(d.Gp), static_cast<float*>(d.Gq), nullptr, nullptr, nullptr, nullptr, 0};
    gpair_one<static_cast<GMode>(MODE), false>(d.n, d.np, sf(st, m, F_NNEW), d.gp_pairs[t], d.gp_sa, par,
                                                static_cast<const float*>(d.W), static_cast<const float*>(d.J2),
                                                d.pmax, static_cast<const float*>(d.Rm), o, wsm + threadIdx.x * 100);
  }
}

// ---- float64 subspace kernels of the batch ---------------------------------------
// Gram blocks C[i][c] = sum_l A_i[l] B_c[l] over the amplitudes, split into
// chunks of kGramChunk amplitudes (partials summed in chunk order by
// bgram_reduce_kernel: deterministic).
enum GrRole { GR_PROJ = 0, GR_GS, GR_LOW, GR_OSC };

template <int ROLE>
__device__ __forceinline__ bool gr_live(const int* st, int m, const BCfg& cfg) {
  if (ROLE == GR_OSC) return sf(st, m, F_STATUS) != BS_UNSTABLE && !cfg.triplet;
  if (!active(st, m)) return false;
  if (ROLE == GR_PROJ) return sf(st, m, F_NNEW) > 0;
  if (ROLE == GR_GS && cfg.pass == 1) return sf(st, m, F_NDIR) > 0 && sf(st, m, F_GS2);
  return sf(st, m, F_NDIR) > 0;
}
template <int ROLE>
__device__ __forceinline__ int gr_rows(const BMol& d, const int* st, int m) {
  if (ROLE == GR_PROJ || ROLE == GR_GS) return sf(st, m, F_S);
  if (ROLE == GR_LOW) return sf(st, m, F_NDIR);
  return d.kk;
}
template <int ROLE>
__device__ __forceinline__ int gr_cols(const BMol& d, const int* st, int m, const BCfg& cfg) {
  if (ROLE == GR_PROJ) return sf(st, m, F_NNEW) * (cfg.rpa ? 2 : 1);
  if (ROLE == GR_OSC) return 3;
  return sf(st, m, F_NDIR);
}
template <int ROLE>
__device__ __forceinline__ const double* gr_a(const BMol& d, int i) {
  if (ROLE == GR_PROJ || ROLE == GR_GS) return d.V + (size_t)i * d.ov;
  if (ROLE == GR_LOW) return d.T + (size_t)i * d.ov;
  return d.Xb + (size_t)i * d.ov;
}
template <int ROLE>
__device__ __forceinline__ const double* gr_b(const BMol& d, const int* st, int m, int c) {
  if (ROLE == GR_PROJ) {
    const int cnt = sf(st, m, F_NNEW), sold = sf(st, m, F_SOLD);
    return c < cnt ? d.S1 + (size_t)(sold + c) * d.ov : d.S2 + (size_t)(sold + c - cnt) * d.ov;
  }
  if (ROLE == GR_OSC) return d.dip + (size_t)c * d.ov;
  return d.T + (size_t)c * d.ov;
}

// The float64 pipe of this part issues one warp instruction per 64 cycles
// per sub-partition whatever the number of active lanes, so only the live
// rows x cols outputs are computed: with P outputs, f = 256 / P threads (a
// power of two, at most 32) share each output over interleaved amplitudes and
// combine by warp shuffles; above 256 outputs each thread takes up to 16.
template <int ROLE>
__global__ void __launch_bounds__(256) bgram_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  __shared__ double As[32][65];
  __shared__ double Bs[32][65];
  const int tid = threadIdx.x;
  RAGGED_PROLOGUE([&](int m) {
    return gr_live<ROLE>(st, m, cfg) ? mols[m].nch * cdiv(gr_rows<ROLE>(mols[m], st, m), 64) : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int rows_all = gr_rows<ROLE>(d, st, m), cols = gr_cols<ROLE>(d, st, m, cfg);
    const int nrb = cdiv(rows_all, 64), lu = u - pref[m];
    const int ch = lu / nrb, rb = lu - ch * nrb;
    const int r0 = rb * 64, rows = min(64, rows_all - r0);
    const int P = rows * cols;
    int f = 1;
    while (f < 32 && P * (2 * f) <= 256) f <<= 1;
    const int ln = tid & (f - 1), og = tid / f, npo = 256 / f;
    int ai[16], bc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int o = og + q * npo;
      ai[q] = o < P ? o / cols : -1;
      bc[q] = o < P ? o - (o / cols) * cols : 0;
    }
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    const long long l0 = (long long)ch * kGramChunk, l1 = min(d.ov, l0 + kGramChunk);
    for (long long lb = l0; lb < l1; lb += 32) {
      __syncthreads();
      for (int e = tid; e < (rows + cols) * 32; e += 256) {
        const int r = e >> 5, ll = e & 31;
        const long long l = lb + ll;
        if (r < rows) As[ll][r] = l < l1 ? gr_a<ROLE>(d, r0 + r)[l] : 0.0;
        else Bs[ll][r - rows] = l < l1 ? gr_b<ROLE>(d, st, m, r - rows)[l] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (ai[q] < 0) break;
        double a = acc[q];
        for (int ll = ln; ll < 32; ll += f) a = fma(As[ll][ai[q]], Bs[ll][bc[q]], a);
        acc[q] = a;
      }
    }
    double* part = d.gpart + ((size_t)ch * 2 + rb) * 4096;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      double a = acc[q];
      for (int o = 1; o < f; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (ai[q] >= 0 && ln == 0) part[ai[q] * 64 + bc[q]] = a;
    }
  }
}

template <int ROLE>
__global__ void __launch_bounds__(256) bgram_reduce_kernel(const BMol* __restrict__ mols,
                                                           const int* __restrict__ st, BCfg cfg) {
  RAGGED_PROLOGUE([&](int m) {
    return gr_live<ROLE>(st, m, cfg)
               ? cdiv((long long)gr_rows<ROLE>(mols[m], st, m) * gr_cols<ROLE>(mols[m], st, m, cfg), 256)
               : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int rows = gr_rows<ROLE>(d, st, m), cols = gr_cols<ROLE>(d, st, m, cfg);
    const int e = (u - pref[m]) * 256 + threadIdx.x;
    if (e >= rows * cols) continue;
    const int i = e / cols, c = e - i * cols;
    const int rb = i >> 6, il = i & 63;
    double s = 0.0;
    for (int ch = 0; ch < d.nch; ++ch) s += d.gpart[((size_t)ch * 2 + rb) * 4096 + il * 64 + c];
    if (ROLE == GR_PROJ) {
      const int cnt = sf(st, m, F_NNEW), sold = sf(st, m, F_SOLD);
      if (c < cnt) d.a1[(size_t)i * d.Smax + sold + c] = s;
      else d.a2[(size_t)i * d.Smax + sold + c - cnt] = s;
    } else if (ROLE == GR_GS) {
      d.tS[(size_t)i * d.maxnew + c] = s;
    } else if (ROLE == GR_LOW) {
      d.G2[(size_t)i * d.maxnew + c] = s;
    } else {
      d.dm[i * 3 + c] = s;
    }
  }
}

// Combinations Y_o = alpha sum_b sum_s coef_b[s][o] X_b[s] + beta Y_o over the
// amplitudes: Ritz vectors and residuals, Gram-Schmidt updates, the appended
// block, the collapsed subspace.  The coefficients go to shared memory; each
// thread owns one amplitude and all outputs.
enum CbRole { CB_RITZ_CIS = 0, CB_RITZ_RPA_R, CB_RITZ_RPA_X, CB_GS, CB_APPEND, CB_COLL };

struct CbJob {
  int nb, rows, nout, ldc;
  const double* X[3];
  const double* coef[3];
  double* Y;
  double alpha, beta;
};

template <int ROLE>
__device__ __forceinline__ int cb_which(const BCfg& cfg) {
  return ROLE == CB_COLL ? (cfg.rpa ? 3 : 2) : 1;
}
template <int ROLE>
__device__ __forceinline__ bool cb_live(const int* st, int m, int pass) {
  if (!active(st, m)) return false;
  if (ROLE == CB_GS) return sf(st, m, F_NDIR) > 0 && (pass == 0 || sf(st, m, F_GS2));
  if (ROLE == CB_APPEND) return sf(st, m, F_NKEEP) > 0;
  if (ROLE == CB_COLL) return sf(st, m, F_COLL) != 0;
  return true;
}

template <int ROLE>
__device__ CbJob cb_job(const BMol& d, const int* st, int m, int which, const BCfg& cfg) {
  CbJob j{};
  const int S = sf(st, m, F_S), kk2 = 2 * d.kk;
  const size_t blk = (size_t)d.Smax * kk2;
  j.alpha = 1.0;
  j.beta = 0.0;
  j.ldc = kk2;
  if (ROLE == CB_RITZ_CIS) {
    j.nb = 2; j.rows = S; j.nout = kk2;
    j.X[0] = d.S1; j.coef[0] = d.coef;
    j.X[1] = d.V; j.coef[1] = d.coef + blk;
    j.Y = d.Xb;
  } else if (ROLE == CB_RITZ_RPA_R) {
    j.nb = 3; j.rows = S; j.nout = kk2;
    j.X[0] = d.S1; j.coef[0] = d.coef;
    j.X[1] = d.V; j.coef[1] = d.coef + blk;
    j.X[2] = d.S2; j.coef[2] = d.coef + 2 * blk;
    j.Y = d.Rb;
  } else if (ROLE == CB_RITZ_RPA_X) {
    j.nb = 1; j.rows = S; j.nout = kk2;
    j.X[0] = d.V; j.coef[0] = d.coef + 3 * blk;
    j.Y = d.Xb;
  } else if (ROLE == CB_GS) {
    j.nb = 1; j.rows = S; j.nout = sf(st, m, F_NDIR); j.ldc = d.maxnew;
    j.X[0] = d.V; j.coef[0] = d.tS;
    j.Y = d.T; j.alpha = -1.0; j.beta = 1.0;
  } else if (ROLE == CB_APPEND) {
    j.nb = 1; j.rows = sf(st, m, F_NDIR); j.nout = sf(st, m, F_NKEEP); j.ldc = d.maxnew;
    j.X[0] = d.T; j.coef[0] = d.Bm;
    j.Y = d.V + (size_t)S * d.ov;
  } else {
    j.nb = 1; j.rows = S; j.nout = sf(st, m, F_NC);
    j.X[0] = which == 0 ? d.V : (which == 1 ? d.S1 : d.S2);
    j.coef[0] = cfg.rpa ? d.E : d.Q;
    j.Y = d.C + (size_t)which * kk2 * d.ov;
  }
  return j;
}

template <int NOUT>
__device__ __forceinline__ void cb_column(const CbJob& j, const double* cs, long long ov, long long l) {
  double acc[NOUT];
#pragma unroll
  for (int o = 0; o < NOUT; ++o) acc[o] = 0.0;
  for (int b = 0; b < j.nb; ++b) {
    const double* X = j.X[b];
    const double* c = cs + (size_t)b * j.rows * NOUT;
    for (int s = 0; s < j.rows; ++s) {
      const double x = X[(size_t)s * ov + l];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) acc[o] = fma(c[s * NOUT + o], x, acc[o]);
    }
  }
  for (int o = 0; o < j.nout; ++o) {
    double* y = j.Y + (size_t)o * ov + l;
    *y = (j.beta != 0.0) ? fma(j.alpha, acc[o], j.beta * *y) : j.alpha * acc[o];
  }
}

template <int ROLE>
__global__ void __launch_bounds__(256) bcombine_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                       BCfg cfg) {
  extern __shared__ double cs[];   // nb x rows x NOUT coefficients (NOUT: nout rounded up to a power of two)
  RAGGED_PROLOGUE([&](int m) {
    return cb_live<ROLE>(st, m, cfg.pass) ? cb_which<ROLE>(cfg) * cdiv(mols[m].ov, kCombChunk) : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int nchk = cdiv(d.ov, kCombChunk);
    const int lu = u - pref[m], which = lu / nchk, ch = lu - which * nchk;
    const CbJob j = cb_job<ROLE>(d, st, m, which, cfg);
    const int NO = j.nout <= 1 ? 1 : j.nout <= 2 ? 2 : j.nout <= 4 ? 4 : j.nout <= 8 ? 8 : (j.nout <= 16 ? 16 : 32);
    __syncthreads();   // the previous unit's reads of cs are done
    for (int idx = threadIdx.x; idx < j.nb * j.rows * NO; idx += blockDim.x) {
      const int b = idx / (j.rows * NO), r = idx - b * (j.rows * NO);
      const int s = r / NO, o = r - s * NO;
      cs[idx] = (o < j.nout) ? j.coef[b][(size_t)s * j.ldc + o] : 0.0;
    }
    __syncthreads();
    const long long l = (long long)ch * kCombChunk + threadIdx.x;
    if (l >= d.ov) continue;
    switch (NO) {
      case 1: cb_column<1>(j, cs, d.ov, l); break;
      case 2: cb_column<2>(j, cs, d.ov, l); break;
      case 4: cb_column<4>(j, cs, d.ov, l); break;
      case 8: cb_column<8>(j, cs, d.ov, l); break;
      case 16: cb_column<16>(j, cs, d.ov, l); break;
      default: cb_column<32>(j, cs, d.ov, l); break;
    }
  }
}

// Ritz vectors and residuals, one thread per amplitude with the subspace
// coefficients in shared memory; only the products that are not zero are
// formed (the float64 pipe is the limit).
//   CIS:  X_j = V q_j, R_j = (A V) q_j - omega_j X_j        -> Xb rows [X | R]
//   TDHF: p_j = V cu_j (X+Y), q_j = V cw_j (X-Y), r1_j = (A+B)V cu_j - omega_j q_j,
//         r2_j = (A-B)V cw_j - omega_j p_j                   -> Xb [p | q], Rb [r1 | r2]
template <int KK, bool RPA>
__device__ __forceinline__ void ritz_column(const BMol& d, int S, const double* cq, const double* om, long long l) {
  const long long ov = d.ov;
  double p[KK], q[KK], a[KK], b[KK];
#pragma unroll
  for (int j = 0; j < KK; ++j) { p[j] = 0.0; q[j] = 0.0; a[j] = 0.0; b[j] = 0.0; }
  for (int s = 0; s < S; ++s) {
    const double v = d.V[(size_t)s * ov + l];
    const double y = d.S1[(size_t)s * ov + l];
    const double* c = cq + (size_t)s * (RPA ? 2 * KK : KK);
    if (RPA) {
      const double z = d.S2[(size_t)s * ov + l];
#pragma unroll
      for (int j = 0; j < KK; ++j) {
        p[j] = fma(c[j], v, p[j]);
        q[j] = fma(c[KK + j], v, q[j]);
        a[j] = fma(c[j], y, a[j]);
        b[j] = fma(c[KK + j], z, b[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < KK; ++j) {
        p[j] = fma(c[j], v, p[j]);
        a[j] = fma(c[j], y, a[j]);
      }
    }
  }
  const int kk = d.kk;
#pragma unroll
  for (int j = 0; j < KK; ++j) {
    if (j >= kk) break;
    if (RPA) {
      d.Xb[(size_t)j * ov + l] = p[j];
      d.Xb[(size_t)(kk + j) * ov + l] = q[j];
      d.Rb[(size_t)j * ov + l] = a[j] - om[j] * q[j];
      d.Rb[(size_t)(kk + j) * ov + l] = b[j] - om[j] * p[j];
    } else {
      d.Xb[(size_t)j * ov + l] = p[j];
      d.Xb[(size_t)(kk + j) * ov + l] = a[j] - om[j] * p[j];
    }
  }
}

template <bool RPA>
__global__ void __launch_bounds__(256) britz_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  __shared__ double cq[kBatchMaxSub * 2 * kBatchMaxRoots];
  __shared__ double om[kBatchMaxRoots];
  RAGGED_PROLOGUE([&](int m) { return active(st, m) ? cdiv(mols[m].ov, kCombChunk) : 0; }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int S = sf(st, m, F_S), kk = d.kk, k = min(kk, S);
    const int KK = kk;   // exact: no float64 FMA on padding
    const int w = RPA ? 2 * KK : KK;
    __syncthreads();   // the previous unit's reads of cq are done
    for (int idx = threadIdx.x; idx < S * w; idx += blockDim.x) {
      const int s = idx / w, c = idx - s * w;
      const int j = RPA ? (c < KK ? c : c - KK) : c;
      const int col = (RPA && c >= KK) ? kk + j : j;   // cu in Q[:, j], cw in Q[:, kk + j]
      cq[idx] = j < k ? d.Q[(size_t)s * 2 * kk + col] : 0.0;
    }
    for (int j = threadIdx.x; j < KK; j += blockDim.x) om[j] = j < k ? d.omega[j] : 0.0;
    __syncthreads();
    const long long l = (long long)(u - pref[m]) * kCombChunk + threadIdx.x;
    if (l >= d.ov) continue;
    switch (KK) {
#define RITZ_CASE(K) \
  case K: ritz_column<K, RPA>(d, S, cq, om, l); break;
      RITZ_CASE(1) RITZ_CASE(2) RITZ_CASE(3) RITZ_CASE(4) RITZ_CASE(5) RITZ_CASE(6) RITZ_CASE(7) RITZ_CASE(8)
      RITZ_CASE(9) RITZ_CASE(10) RITZ_CASE(11) RITZ_CASE(12) RITZ_CASE(13) RITZ_CASE(14) RITZ_CASE(15)
      default: ritz_column<16, RPA>(d, S, cq, om, l); break;
#undef RITZ_CASE
    }
  }
}

// second Gram-Schmidt pass only where the first removed more than half of a
// direction's norm^2 (unit rows in, norms below 0.7 out): "twice is enough"
__global__ void bgs_check_kernel(const BMol* __restrict__ mols, int* __restrict__ st, BCfg cfg) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= cfg.nmol || !active(st, m)) return;
  const BMol& d = mols[m];
  const int nd = sf(st, m, F_NDIR);
  int need = 0;
  for (int j = 0; j < nd; ++j) need |= !(d.tn[j] >= 0.7);
  st[m * kSt + F_GS2] = need;
}

// Row 2-norms, one CTA per row (fixed reduction order): residual rows (CIS:
// A X - omega X in Xb rows kk..; TDHF: r1, r2 in Rb) or the new directions.
enum RnRole { RN_RES = 0, RN_T };

template <int ROLE>
__global__ void __launch_bounds__(256) bnorm_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  __shared__ double red[8];
  RAGGED_PROLOGUE([&](int m) {
    if (!active(st, m)) return 0;
    return ROLE == RN_RES ? (cfg.rpa ? 2 : 1) * mols[m].kk : sf(st, m, F_NDIR);
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int j = u - pref[m];
    const double* x = ROLE == RN_T ? d.T + (size_t)j * d.ov
                                   : (cfg.rpa ? d.Rb + (size_t)j * d.ov : d.Xb + (size_t)(d.kk + j) * d.ov);
    double s = 0.0;
    for (long long l = threadIdx.x; l < d.ov; l += blockDim.x) s = fma(x[l], x[l], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      (ROLE == RN_T ? d.tn : d.nrm)[j] = sqrt(t);
    }
  }
}

// New directions: T_s = r_root / (omega_root - de), the denominator's
// magnitude clamped to >= 1e-4 eV and inverted in float32 (a search direction
// only; it is orthonormalised in float64 next); then scaled to unit rows.
template <bool SCALE>
__global__ void __launch_bounds__(256) bprecond_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                       BCfg cfg) {
  RAGGED_PROLOGUE([&](int m) { return active(st, m) ? sf(st, m, F_NDIR) * cdiv(mols[m].ov, 2048) : 0; }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int nchk = cdiv(d.ov, 2048), lu = u - pref[m];
    const int s = lu / nchk, ch = lu - s * nchk;
    double* t = d.T + (size_t)s * d.ov;
    const long long l0 = (long long)ch * 2048, l1 = min(d.ov, l0 + 2048);
    if (SCALE) {
      const double nr = d.tn[s];
      const double sc = nr > 0.0 ? 1.0 / nr : 0.0;
      for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) t[l] *= sc;
    } else {
      const int code = d.slot[s], root = code >> 1, kind = code & 1;
      const double* r = cfg.rpa ? d.Rb + (size_t)(kind * d.kk + root) * d.ov : d.Xb + (size_t)(d.kk + root) * d.ov;
      const float w = static_cast<float>(d.omega[root]);
      const double* sh = sf(st, m, F_NOSHIFT) ? nullptr : d.shift;
      for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
        float den = w - static_cast<float>(de_of(d, l));
        if (sh) den -= static_cast<float>(sh[l]);
        if (fabsf(den) < 1e-4f) den = (den < 0.0f) ? -1e-4f : 1e-4f;
        t[l] = r[l] * static_cast<double>(__frcp_rn(den));
      }
    }
  }
}

// collapsed subspace back into V, A V (and (A-B) V): rows [0, nc)
__global__ void __launch_bounds__(256) bcopy_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  RAGGED_PROLOGUE([&](int m) {
    return (active(st, m) && sf(st, m, F_COLL)) ? (cfg.rpa ? 3 : 2) * sf(st, m, F_NC) * cdiv(mols[m].ov, 4096) : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int nchk = cdiv(d.ov, 4096), nc = sf(st, m, F_NC), lu = u - pref[m];
    const int which = lu / (nc * nchk), rem = lu - which * nc * nchk;
    const int row = rem / nchk, ch = rem - row * nchk;
    double* dst = (which == 0 ? d.V : (which == 1 ? d.S1 : d.S2)) + (size_t)row * d.ov;
    const double* src = d.C + (size_t)(which * 2 * d.kk + row) * d.ov;
    const long long l0 = (long long)ch * 4096, l1 = min(d.ov, l0 + 4096);
    for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) dst[l] = src[l];
  }
}

// ---- per-molecule small kernels (one CTA per molecule) ----------------------------
// Rayleigh-Ritz step.  CIS: the lowest eigenpairs of the projected matrix
// (upper triangle of a1 valid); TDHF: a- = L L^T, M = L^T a+ L, M z = omega^2 z,
// X+Y = V L z / sqrt(omega), X-Y = V a+ (X+Y)~ / omega.  Writes omega and the
// coefficient blocks of the Ritz-vector and residual combinations.
__global__ void __launch_bounds__(1024) beig_kernel(const BMol* __restrict__ mols, int* __restrict__ st, BCfg cfg) {
  const int m = blockIdx.x;
  if (m >= cfg.nmol || !active(st, m)) return;
  const BMol& d = mols[m];
  const int S = sf(st, m, F_S), kk = d.kk, kk2 = 2 * kk, k = min(kk, S), ld = d.Smax;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t blk = (size_t)d.Smax * kk2;
  __shared__ int flag;
  if (!cfg.rpa) {
    for (int idx = tid; idx < S * S; idx += nt) {
      const int i = idx / S, j = idx - i * S;
      d.Mb[(size_t)i * ld + j] = d.a1[(size_t)min(i, j) * ld + max(i, j)];
    }
    __syncthreads();
    const int kq = min(S, kk2);
    syevk_body<true>(S, kq, d.Mb, ld, d.wts, d.Q, kk2, d.syw, nullptr);
    __syncthreads();
    if (tid == 0) st[m * kSt + F_KQ] = kq;
    for (int j = tid; j < kk; j += nt) d.omega[j] = j < k ? d.wts[j] : 0.0;
    __syncthreads();
    for (int idx = tid; idx < S * kk2; idx += nt) {
      const int s = idx / kk2, o = idx - s * kk2;
      const int r = o < kk ? o : o - kk;
      const double q = r < k ? d.Q[(size_t)s * kk2 + r] : 0.0;
      d.coef[idx] = o < kk ? 0.0 : q;                                       // A V
      d.coef[blk + idx] = o < kk ? q : (r < k ? -d.omega[r] * q : 0.0);     // V
    }
    return;
  }
  // TDHF
  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, j = idx - i * S;
    const size_t up = (size_t)min(i, j) * ld + max(i, j);
    d.Lb[(size_t)i * ld + j] = d.a2[up];
    d.Mb[(size_t)i * ld + j] = d.a1[up];
  }
  if (tid == 0) flag = 0;
  __syncthreads();
  cholesky_body<true>(S, d.Lb, ld, &flag);
  __syncthreads();
  if (flag) {
    if (tid == 0) st[m * kSt + F_STATUS] = BS_UNSTABLE;
    return;
  }
  // Pb = L^T a+, Nb = Pb L
  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, j = idx - i * S;
    double acc = 0.0;
    for (int q = i; q < S; ++q) acc = fma(d.Lb[(size_t)q * ld + i], d.Mb[(size_t)q * ld + j], acc);
    d.Pb[(size_t)i * ld + j] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, j = idx - i * S;
    double acc = 0.0;
    for (int q = j; q < S; ++q) acc = fma(d.Pb[(size_t)i * ld + q], d.Lb[(size_t)q * ld + j], acc);
    d.Nb[(size_t)i * ld + j] = acc;
  }
  __syncthreads();
  syevk_body<true>(S, k, d.Nb, ld, d.wts, d.E, kk2, d.syw, nullptr);
  __syncthreads();
  if (tid == 0) {
    int bad = 0;
    for (int j = 0; j < k; ++j) bad |= !(d.wts[j] > 0.0);
    flag = bad;
  }
  __syncthreads();
  if (flag) {
    if (tid == 0) st[m * kSt + F_STATUS] = BS_UNSTABLE;
    return;
  }
  for (int j = tid; j < kk; j += nt) d.omega[j] = j < k ? sqrt(d.wts[j]) : 0.0;
  __syncthreads();
  // cu = L z / sqrt(omega) in Q[:, 0..kk), cw = a+ cu / omega in Q[:, kk..)
  for (int idx = tid; idx < S * k; idx += nt) {
    const int i = idx / k, j = idx - i * k;
    double acc = 0.0;
    for (int q = 0; q <= i; ++q) acc = fma(d.Lb[(size_t)i * ld + q], d.E[(size_t)q * kk2 + j], acc);
    d.Q[(size_t)i * kk2 + j] = acc / sqrt(d.omega[j]);
  }
  __syncthreads();
  for (int idx = tid; idx < S * k; idx += nt) {
    const int i = idx / k, j = idx - i * k;
    double acc = 0.0;
    for (int q = 0; q < S; ++q) acc = fma(d.Mb[(size_t)i * ld + q], d.Q[(size_t)q * kk2 + j], acc);
    d.Q[(size_t)i * kk2 + kk + j] = acc / d.omega[j];
  }
  __syncthreads();
  for (int idx = tid; idx < S * kk2; idx += nt) {
    const int s = idx / kk2, o = idx - s * kk2;
    const int r = o < kk ? o : o - kk;
    const bool ok = r < k;
    const double cu = ok ? d.Q[(size_t)s * kk2 + r] : 0.0;
    const double cw = ok ? d.Q[(size_t)s * kk2 + kk + r] : 0.0;
    const double om = ok ? d.omega[r] : 0.0;
    d.coef[idx] = o < kk ? cu : 0.0;                       // (A+B) V
    d.coef[blk + idx] = o < kk ? -om * cw : -om * cu;      // V
    d.coef[2 * blk + idx] = o < kk ? 0.0 : cw;             // (A-B) V
    d.coef[3 * blk + idx] = o < kk ? cu : cw;              // V -> X+Y, X-Y
  }
}

// Loewdin factor of the Gram matrix G (n x n, row stride ldg): eigenvalues
// above thresh * max(lambda_max, 1) kept from the largest down; B[s][q] =
// Q[s][j_q] / sqrt(lambda_{j_q}) (row stride ldb); returns the count.  One
// CTA, matrices up to 32 x 32 in shared memory.
__device__ int lowdin_block(int nd, const double* G, int ldg, double* B, int ldb) {
  __shared__ double As[32 * 33], Vs[32 * 33], scr[64];
  __shared__ double lam[32];
  __shared__ int ord[32], nkeep;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < nd * nd; idx += nt) {
    const int i = idx / nd, j = idx - i * nd;
    As[i * 33 + j] = 0.5 * (G[(size_t)i * ldg + j] + G[(size_t)j * ldg + i]);
  }
  __syncthreads();
  jacobi_sweeps(nd, As, 33, Vs, 33, scr, 64);
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < nd; ++j) { lam[j] = As[j * 33 + j]; ord[j] = j; }
    // descending eigenvalues (insertion sort, ties by index)
    for (int a = 1; a < nd; ++a) {
      const int x = ord[a];
      int b = a - 1;
      while (b >= 0 && lam[ord[b]] < lam[x]) { ord[b + 1] = ord[b]; --b; }
      ord[b + 1] = x;
    }
    const double lmax = fmax(nd > 0 ? lam[ord[0]] : 1.0, 1.0);
    int c = 0;
    while (c < nd && lam[ord[c]] > kLowdinThresh * lmax) ++c;
    nkeep = c;
  }
  __syncthreads();
  const int nk = nkeep;
  for (int idx = tid; idx < nd * nk; idx += nt) {
    const int s = idx / nk, q = idx - s * nk;
    const int j = ord[q];
    B[(size_t)s * ldb + q] = Vs[s * 33 + j] / sqrt(lam[j]);
  }
  __syncthreads();
  return nk;
}

// Convergence and restart decisions after the residual norms: converged
// roots drop out; each unconverged root contributes its preconditioned
// residual (TDHF: both); when the new block would overflow the subspace it
// collapses first (CIS: onto the 2k lowest Ritz vectors; TDHF: onto an
// orthonormal basis of span{X+Y, X-Y}, with the projected matrices rotated
// along).
__global__ void __launch_bounds__(256) bdecide_kernel(const BMol* __restrict__ mols, int* __restrict__ st, BCfg cfg) {
  const int m = blockIdx.x;
  if (m >= cfg.nmol || !active(st, m)) return;
  const BMol& d = mols[m];
  const int S = sf(st, m, F_S), kk = d.kk, kk2 = 2 * kk, k = min(kk, S), ld = d.Smax;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int sh_ndir, sh_coll, sh_nc, sh_done;
  if (tid == 0) {
    const int it = sf(st, m, F_ITER) + 1;
    st[m * kSt + F_ITER] = it;
    bool all = (k == kk);
    int nd = 0;
    for (int j = 0; j < k; ++j) {
      const double r = cfg.rpa ? fmax(d.nrm[j], d.nrm[kk + j]) : d.nrm[j];
      if (!(r <= cfg.tol)) {
        all = false;
        d.slot[nd++] = 2 * j;
        if (cfg.rpa) d.slot[nd++] = 2 * j + 1;
      }
    }
    // learned shift dropped when the largest residual has not fallen by 10 %
    // over the last five iterations (the plain preconditioner takes over)
    if (d.shift && !sf(st, m, F_NOSHIFT)) {
      double mr = 0.0;
      for (int j = 0; j < k; ++j) mr = fmax(mr, cfg.rpa ? fmax(d.nrm[j], d.nrm[kk + j]) : d.nrm[j]);
      d.rhist[it & 7] = mr;
      if (it > 5 && mr > 0.9 * d.rhist[(it - 5) & 7]) st[m * kSt + F_NOSHIFT] = 1;
    }
    int done = 0;
    if (all) done = BS_CONVERGED;
    else if (it >= cfg.max_iter) done = BS_MAXITER;
    sh_done = done;
    sh_ndir = nd;
    sh_coll = (!done && S + nd > d.Smax) ? 1 : 0;
    sh_nc = cfg.rpa ? 0 : sf(st, m, F_KQ);
  }
  __syncthreads();
  if (sh_done) {
    if (tid == 0) {
      st[m * kSt + F_STATUS] = sh_done;
      st[m * kSt + F_NDIR] = 0;
    }
    return;
  }
  int nc = S;
  if (sh_coll) {
    if (!cfg.rpa) {
      nc = sh_nc;
      for (int idx = tid; idx < nc * nc; idx += nt) {
        const int i = idx / nc, j = idx - i * nc;
        d.a1[(size_t)i * ld + j] = (i == j) ? d.wts[i] : 0.0;
      }
    } else {
      // Gram of the 2k coefficient columns [cu | cw], Loewdin basis E = [cu cw] B
      const int c2 = 2 * k;
      for (int idx = tid; idx < c2 * c2; idx += nt) {
        const int a = idx / c2, b = idx - a * c2;
        const int ca = a < k ? a : kk + a - k, cb = b < k ? b : kk + b - k;
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc = fma(d.Q[(size_t)s * kk2 + ca], d.Q[(size_t)s * kk2 + cb], acc);
        d.G2[(size_t)a * d.maxnew + b] = acc;
      }
      __syncthreads();
      nc = lowdin_block(c2, d.G2, d.maxnew, d.Bm, d.maxnew);   // Bm[c][q], c < 2k, q < nc
      for (int idx = tid; idx < S * nc; idx += nt) {
        const int s = idx / nc, q = idx - s * nc;
        double acc = 0.0;
        for (int c = 0; c < c2; ++c) {
          const int cc = c < k ? c : kk + c - k;
          acc = fma(d.Q[(size_t)s * kk2 + cc], d.Bm[(size_t)c * d.maxnew + q], acc);
        }
        d.E[(size_t)s * kk2 + q] = acc;
      }
      __syncthreads();
      // a+' = E^T a+ E, a-' = E^T a- E (full nc x nc)
      for (int pass = 0; pass < 2; ++pass) {
        double* a = pass ? d.a2 : d.a1;
        for (int idx = tid; idx < S * nc; idx += nt) {
          const int s = idx / nc, q = idx - s * nc;
          double acc = 0.0;
          for (int t = 0; t < S; ++t)
            acc = fma(a[(size_t)min(s, t) * ld + max(s, t)], d.E[(size_t)t * kk2 + q], acc);
          d.Pb[(size_t)s * ld + q] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < nc * nc; idx += nt) {
          const int p = idx / nc, q = idx - p * nc;
          double acc = 0.0;
          for (int s = 0; s < S; ++s) acc = fma(d.E[(size_t)s * kk2 + p], d.Pb[(size_t)s * ld + q], acc);
          d.Nb[(size_t)p * ld + q] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < nc * nc; idx += nt) {
          const int p = idx / nc, q = idx - p * nc;
          a[(size_t)p * ld + q] = d.Nb[(size_t)p * ld + q];
        }
        __syncthreads();
      }
    }
  }
  if (tid == 0) {
    int nd = min(sh_ndir, d.Smax - nc);
    st[m * kSt + F_COLL] = sh_coll;
    st[m * kSt + F_NC] = nc;
    st[m * kSt + F_NDIR] = nd > 0 ? nd : 0;
    if (nd <= 0) st[m * kSt + F_STATUS] = BS_STALLED;
  }
}

// Loewdin orthonormalisation of the new directions (after Gram-Schmidt):
// coefficients of the kept combinations for the append step.
__global__ void __launch_bounds__(256) blowdin_kernel(const BMol* __restrict__ mols, int* __restrict__ st, BCfg cfg) {
  const int m = blockIdx.x;
  if (m >= cfg.nmol || !active(st, m)) return;
  const BMol& d = mols[m];
  const int nd = sf(st, m, F_NDIR);
  if (nd <= 0) return;
  const int nk = lowdin_block(nd, d.G2, d.maxnew, d.Bm, d.maxnew);
  if (threadIdx.x == 0) {
    st[m * kSt + F_NKEEP] = nk;
    if (nk == 0) st[m * kSt + F_STATUS] = BS_STALLED;
  }
}

// S := the collapsed size (after the collapsed vectors are copied back)
__global__ void bcollapse_apply_kernel(int* __restrict__ st, BCfg cfg) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= cfg.nmol || !active(st, m) || !sf(st, m, F_COLL)) return;
  st[m * kSt + F_S] = sf(st, m, F_NC);
  st[m * kSt + F_COLL] = 0;
}

// the appended block becomes the next products' input; count the molecules
// still active (one CTA)
__global__ void __launch_bounds__(1024) badvance_kernel(int* __restrict__ st, BCfg cfg, int* __restrict__ nactive) {
  __shared__ int red[32];
  int cnt = 0;
  for (int m = threadIdx.x; m < cfg.nmol; m += blockDim.x) {
    int* s = st + m * kSt;
    if (s[F_STATUS] == BS_ACTIVE) {
      s[F_SOLD] = s[F_S];
      s[F_S] += s[F_NKEEP];
      s[F_NNEW] = s[F_NKEEP];
      s[F_PROD] += s[F_NKEEP];
      ++cnt;
    } else {
      s[F_NNEW] = 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *nactive = t;
  }
}

// unit start vectors: V[j] = e_{gidx[j]}
__global__ void __launch_bounds__(256) bguess_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                     BCfg cfg, const long long* __restrict__ gidx, int gld) {
  RAGGED_PROLOGUE([&](int m) { return sf(st, m, F_NNEW) * cdiv(mols[m].ov, 4096); }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int nchk = cdiv(d.ov, 4096), lu = u - pref[m];
    const int j = lu / nchk, ch = lu - j * nchk;
    const long long g = gidx[(size_t)m * gld + j];
    double* x = d.V + (size_t)j * d.ov;
    const long long l0 = (long long)ch * 4096, l1 = min(d.ov, l0 + 4096);
    for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) x[l] = (l == g) ? 1.0 : 0.0;
  }
}

// learned guess: the nguess scored pairs of highest predicted weight (output
// 1; ties to the lower gap, i.e. the earlier pair), one CTA per molecule;
// pairs, rows and out concatenated over the molecules
__global__ void __launch_bounds__(256) bselect_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                      BCfg cfg, const long long* __restrict__ pairs,
                                                      const int* __restrict__ row0, const int* __restrict__ nrow,
                                                      const float* __restrict__ out, long long* __restrict__ gidx,
                                                      int gld) {
  const int m = blockIdx.x;
  if (m >= cfg.nmol) return;
  __shared__ float bv[256];
  __shared__ int bi[256];
  __shared__ int taken[32];
  const int r0 = row0[m], nr = nrow[m], ng = sf(st, m, F_NNEW);
  for (int j = 0; j < ng; ++j) {
    float best = -INFINITY;
    int bq = 0x7fffffff;
    for (int q = threadIdx.x; q < nr; q += blockDim.x) {
      bool used = false;
      for (int t = 0; t < j; ++t) used |= taken[t] == q;
      if (used) continue;
      const float v = out[(size_t)(r0 + q) * kMlpOutputs + 1];
      if (v > best || (v == best && q < bq)) { best = v; bq = q; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bq;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const float v2 = bv[threadIdx.x + o];
        const int i2 = bi[threadIdx.x + o];
        if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
          bv[threadIdx.x] = v2;
          bi[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      taken[j] = bi[0];
      gidx[(size_t)m * gld + j] = pairs[r0 + bi[0]];
    }
    __syncthreads();
  }
}

// learned shift of every scored pair (output 0), zero elsewhere (zeroed before)
__global__ void __launch_bounds__(256) bshift_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                     BCfg cfg, const long long* __restrict__ pairs,
                                                     const int* __restrict__ row0, const int* __restrict__ nrow,
                                                     const float* __restrict__ out) {
  RAGGED_PROLOGUE([&](int m) { return mols[m].shift ? cdiv(nrow[m], 256) : 0; }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int q = (u - pref[m]) * 256 + threadIdx.x;
    if (q >= nrow[m]) continue;
    const int r = row0[m] + q;
    d.shift[pairs[r]] = static_cast<double>(out[(size_t)r * kMlpOutputs]);
  }
}

// oscillator strengths from the transition dipoles dm (kk x 3, Angstrom)
__global__ void bosc_kernel(const BMol* __restrict__ mols, const int* __restrict__ st, BCfg cfg) {
  const int m = blockIdx.x;
  if (m >= cfg.nmol) return;
  const BMol& d = mols[m];
  for (int j = threadIdx.x; j < d.kk; j += blockDim.x) {
    double s2 = 0.0;
    if (!cfg.triplet && sf(st, m, F_STATUS) != BS_UNSTABLE)
      for (int x = 0; x < 3; ++x) {
        const double dv = d.dm[j * 3 + x] * (1.4142135623730951 / kBohrA);
        s2 += dv * dv;
      }
    d.osc[j] = (2.0 / 3.0) * (d.omega[j] / kHartreeEV) * s2;
  }
}

}  // namespace

namespace {

// results of every molecule into one block: omega, residual, f (kk each)
__global__ void bresults_kernel(const BMol* __restrict__ mols, const int* __restrict__ st, BCfg cfg,
                                double* __restrict__ out, int ldo) {
  const int m = blockIdx.x;
  if (m >= cfg.nmol) return;
  const BMol& d = mols[m];
  for (int j = threadIdx.x; j < d.kk; j += blockDim.x) {
    out[(size_t)m * ldo + j] = d.omega[j];
    out[(size_t)m * ldo + d.kk + j] = cfg.rpa ? fmax(d.nrm[j], d.nrm[d.kk + j]) : d.nrm[j];
    out[(size_t)m * ldo + 2 * d.kk + j] = d.osc[j];
  }
}

// the kept amplitudes: U = X (CIS) or X+Y, Wv = X (CIS) or X-Y
__global__ void __launch_bounds__(256) bkeep_kernel(const BMol* __restrict__ mols, const int* __restrict__ st,
                                                    BCfg cfg) {
  RAGGED_PROLOGUE([&](int m) {
    return sf(st, m, F_STATUS) != BS_UNSTABLE ? 2 * mols[m].kk * cdiv(mols[m].ov, 4096) : 0;
  }) {
    const int m = find_mol(pref, cfg.nmol, u);
    const BMol& d = mols[m];
    const int nchk = cdiv(d.ov, 4096), lu = u - pref[m];
    const int row = lu / nchk, ch = lu - row * nchk;
    const int which = row / d.kk, j = row - which * d.kk;
    const double* src = d.Xb + (size_t)((cfg.rpa && which) ? d.kk + j : j) * d.ov;
    double* dst = (which ? d.Wv : d.U) + (size_t)j * d.ov;
    const long long l0 = (long long)ch * 4096, l1 = min(d.ov, l0 + 4096);
    for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) dst[l] = src[l];
  }
}

#define BATCH_LAUNCHED() XS_CUDA(cudaGetLastError())

// Device arenas and graph of the lock-step solver, kept in the context between
// solves (buffers only grow).
struct BatchWork {
  DevBuf<double> dsub;     // float64 subspace arena
  DevBuf<float> fprod;     // float32 product arena
  DevBuf<double> dprod;    // float64 product arena
  DevBuf<int> islot;       // slot maps
  DevBuf<BMol> dmols;
  DevBuf<int> dst;
  DevBuf<long long> gidx;
  DevBuf<double> results;
  DevBuf<int> nact;
  // learned guess: features, network activations, outputs, pair lists
  FeatureWork fw;
  DevBuf<long long> dpairs, lpairs;
  DevBuf<float> F, out;
  DevBuf<int> lrow;
  std::vector<DevBuf<float>> Z, H;
  MlpOperands mo;   // the network's tensor-core operand pairs
  int* hnact = nullptr;    // page-locked copy of the active count
  BatchWork() = default;
  BatchWork(const BatchWork&) = delete;
  BatchWork& operator=(const BatchWork&) = delete;
  ~BatchWork() {
    if (hnact) cudaFreeHost(hnact);
  }
};

constexpr int kGridCTAs = 152 * 4;   // persistent grids: 4 CTAs per SM
// learned guess: candidate pairs (lowest orbital-energy gaps) scored per
// molecule, as in the one-molecule solver; network rows per forward chunk
constexpr long long kLearnedPairs = 16384;
constexpr int kForwardRows = 1 << 20;

template <typename T>
void ensure_product_operands(Ctx& c, DevMol& m) {
  if (sizeof(T) != 4) return;
  cudaStream_t s = c.stream;
  if (!m.Wf.get()) {
    m.Wf.alloc((size_t)m.np * m.np);
    convert_d2f(s, (long long)m.np * m.np, m.W.get(), m.Wf.get());
  }
  if (!m.CTf.get()) {
    m.CTf.alloc((size_t)m.n * m.n);
    convert_d2f(s, (long long)m.n * m.n, m.CT.get(), m.CTf.get());
  }
}

template <int ROLE>
void set_smem_attr(const void* fn, int bytes) {
  static const bool once = [&] {
    XS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return true;
  }();
  (void)once;
}

// one Davidson iteration of the whole batch (the captured sequence)
template <typename T, int MODE>
int enqueue_iteration(cudaStream_t s, const BMol* mols, int* st, const BCfg& cfg, const double* par, int* nact,
                      int* hnact) {
  const int kCombSmem = 3 * cfg.smax * 32 * 8;
  const size_t kEigSmem = sizeof(double) * syevk_work_doubles(cfg.smax);
  int launches = 0;
  auto L = [&]() { BATCH_LAUNCHED(); ++launches; };
  // products of the appended vectors
  if (sizeof(T) == 4) { bconvert_kernel<<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L(); }
  bgemm_kernel<T, R_P1><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bgemm_kernel<T, R_P2><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  if (cfg.coulomb) {
    bpack_kernel<T><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
    bgemm_kernel<T, R_J2><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  }
  if (sizeof(T) == 4) {
    bgpair_kernel<MODE><<<kGridCTAs, 256, sizeof(float) * 100 * 256, s>>>(mols, st, cfg, par); L();
  } else {
    bgtile_kernel<T, MODE><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg, par); L();
  }
  bgemm_kernel<T, R_B1><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bgemm_kernel<T, R_B2><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  // projected matrices and the Rayleigh-Ritz step
  bgram_kernel<GR_PROJ><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bgram_reduce_kernel<GR_PROJ><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  beig_kernel<<<cfg.nmol, 1024, kEigSmem, s>>>(mols, st, cfg); L();
  if (!cfg.rpa) {
    britz_kernel<false><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  } else {
    britz_kernel<true><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  }
  bnorm_kernel<RN_RES><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bdecide_kernel<<<cfg.nmol, 256, 0, s>>>(mols, st, cfg); L();
  // new directions, collapse, orthonormalisation, append
  bprecond_kernel<false><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bcombine_kernel<CB_COLL><<<kGridCTAs, 256, kCombSmem, s>>>(mols, st, cfg); L();
  bcopy_kernel<<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bcollapse_apply_kernel<<<cdiv(cfg.nmol, 256), 256, 0, s>>>(st, cfg); L();
  bnorm_kernel<RN_T><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bprecond_kernel<true><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  for (int pass = 0; pass < 2; ++pass) {
    BCfg cp = cfg;
    cp.pass = pass;
    bgram_kernel<GR_GS><<<kGridCTAs, 256, 0, s>>>(mols, st, cp); L();
    bgram_reduce_kernel<GR_GS><<<kGridCTAs, 256, 0, s>>>(mols, st, cp); L();
    bcombine_kernel<CB_GS><<<kGridCTAs, 256, kCombSmem, s>>>(mols, st, cp); L();
    if (pass == 0) {
      bnorm_kernel<RN_T><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
      bgs_check_kernel<<<cdiv(cfg.nmol, 256), 256, 0, s>>>(mols, st, cfg); L();
    }
  }
  bgram_kernel<GR_LOW><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  bgram_reduce_kernel<GR_LOW><<<kGridCTAs, 256, 0, s>>>(mols, st, cfg); L();
  blowdin_kernel<<<cfg.nmol, 256, 0, s>>>(mols, st, cfg); L();
  bcombine_kernel<CB_APPEND><<<kGridCTAs, 256, kCombSmem, s>>>(mols, st, cfg); L();
  badvance_kernel<<<1, 1024, 0, s>>>(st, cfg, nact); L();
  XS_CUDA(cudaMemcpyAsync(hnact, nact, sizeof(int), cudaMemcpyDeviceToHost, s));
  return launches;
}

void set_attributes() {
  constexpr int kCombSmem = 3 * kBatchMaxSub * 32 * 8;
  static const bool eig_attr = [] {
    XS_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(beig_kernel),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sizeof(double) * syevk_work_doubles(kBatchMaxSub))));
    return true;
  }();
  (void)eig_attr;
  static const bool pair_attr = [] {
    for (const void* f : {reinterpret_cast<const void*>(bgpair_kernel<G_CIS>),
                          reinterpret_cast<const void*>(bgpair_kernel<G_RPA>),
                          reinterpret_cast<const void*>(bgpair_kernel<G_CIS_T>),
                          reinterpret_cast<const void*>(bgpair_kernel<G_RPA_T>)})
      XS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(float) * 100 * 256)));
    return true;
  }();
  (void)pair_attr;
  set_smem_attr<CB_RITZ_CIS>(reinterpret_cast<const void*>(bcombine_kernel<CB_RITZ_CIS>), kCombSmem);
  set_smem_attr<CB_RITZ_RPA_R>(reinterpret_cast<const void*>(bcombine_kernel<CB_RITZ_RPA_R>), kCombSmem);
  set_smem_attr<CB_RITZ_RPA_X>(reinterpret_cast<const void*>(bcombine_kernel<CB_RITZ_RPA_X>), kCombSmem);
  set_smem_attr<CB_GS>(reinterpret_cast<const void*>(bcombine_kernel<CB_GS>), kCombSmem);
  set_smem_attr<CB_APPEND>(reinterpret_cast<const void*>(bcombine_kernel<CB_APPEND>), kCombSmem);
  set_smem_attr<CB_COLL>(reinterpret_cast<const void*>(bcombine_kernel<CB_COLL>), kCombSmem);
}

struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  ~GraphGuard() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
  }
};

template <typename T, int MODE>
int capture_iteration(cudaStream_t s, const BMol* mols, int* st, const BCfg& cfg, const double* par, int* nact,
                      int* hnact, GraphGuard& gg) {
  XS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int launches = 0;
  try {
    launches = enqueue_iteration<T, MODE>(s, mols, st, cfg, par, nact, hnact);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  XS_CUDA(cudaStreamEndCapture(s, &gg.g));
  XS_CUDA(cudaGraphInstantiate(&gg.e, gg.g, 0));
  return launches;
}

template <typename T>
int capture_mode(cudaStream_t s, const BMol* mols, int* st, const BCfg& cfg, const double* par, int* nact,
                 int* hnact, GraphGuard& gg) {
  switch (cfg.mode) {
    case G_CIS: return capture_iteration<T, G_CIS>(s, mols, st, cfg, par, nact, hnact, gg);
    case G_RPA: return capture_iteration<T, G_RPA>(s, mols, st, cfg, par, nact, hnact, gg);
    case G_CIS_T: return capture_iteration<T, G_CIS_T>(s, mols, st, cfg, par, nact, hnact, gg);
    default: return capture_iteration<T, G_RPA_T>(s, mols, st, cfg, par, nact, hnact, gg);
  }
}

size_t up32(size_t x) { return (x + 31) / 32 * 32; }

template <typename T>
void solve_group(Ctx& c, BatchWork& bw, const xs_ex_opts& opt, int first, int count, std::vector<SolveStats>& st,
                 std::vector<int>& rcs, long long* graph_launches) {
  cudaStream_t s = c.stream;
  const bool rpa = opt.method == XS_TDHF, triplet = opt.spin == XS_TRIPLET;
  const bool learned = opt.guess == XS_GUESS_LEARNED && !triplet && c.mlp && c.mlp->ready;
  BCfg cfg{};
  cfg.nmol = count;
  cfg.rpa = rpa;
  cfg.triplet = triplet;
  cfg.coulomb = !triplet;
  cfg.mode = gmode(rpa, triplet);
  cfg.max_iter = opt.max_iter > 0 ? opt.max_iter : 200;
  cfg.tol = (opt.precision == XS_MIXED) ? std::max(opt.tol, kMixedResidualFloor) : opt.tol;

  // sizes and arena offsets
  std::vector<BMol> h(count);
  std::vector<size_t> off_sub(count), off_prod(count), off_slot(count);
  size_t nsub = 0, nprod = 0, nslot = 0;
  std::vector<std::vector<long long>> guess(count);
  int gld = 1;
  for (int q = 0; q < count; ++q) {
    DevMol& m = c.mols[first + q];
    ensure_product_operands<T>(c, m);
    if (!triplet) mo_dipoles(c, m);
    BMol& d = h[q];
    std::memset(&d, 0, sizeof(d));
    d.n = m.n; d.o = m.o; d.v = m.v; d.np = m.np; d.natoms = m.L.natoms;
    d.ov = (long long)m.o * m.v;
    if (d.v > d.o) throw Error(XS_EINVAL, "batched solve: nvir > nocc (not a neutral H/C/N/O molecule)");
    d.kk = static_cast<int>(std::min<long long>(opt.nroots, d.ov));
    d.maxnew = rpa ? 2 * d.kk : d.kk;
    const int nguess = static_cast<int>(std::min<long long>(d.ov, std::max(2 * d.kk, d.kk + 2)));
    d.pmax = std::max(d.maxnew, nguess);
    int smax = opt.max_subspace > 0 ? opt.max_subspace : std::max(48, (rpa ? 16 : 10) * d.kk);
    smax = std::min(smax, kBatchMaxSub);
    smax = static_cast<int>(std::min<long long>(smax, d.ov));
    smax = std::max(smax, static_cast<int>(std::min<long long>(d.ov, nguess + 2 * d.kk)));
    if (smax > kBatchMaxSub) throw Error(XS_EINVAL, "batched solve: subspace above 128 vectors");
    d.Smax = smax;
    d.nch = cdiv(d.ov, kGramChunk);
    d.ntr = m.gb_nrows; d.ntc = m.gb_ncols;
    const size_t ov = (size_t)d.ov, S = (size_t)smax, k2 = 2 * (size_t)d.kk, mn = (size_t)d.maxnew;
    off_sub[q] = nsub;
    nsub += up32(S * ov) * (rpa ? 3 : 2) + up32(k2 * ov) * (rpa ? 2 : 1) + up32(mn * ov) +
            up32((rpa ? 3 : 2) * k2 * ov) + up32(S * S) * 6 + up32(S * k2) * 6 + up32(S * mn) + up32(mn * mn) * 2 +
            up32(S) + up32(d.kk) * 3 + up32(k2) + up32(mn) + up32(3 * (size_t)d.kk) + up32((size_t)d.nch * 2 * 4096) +
            up32(syevk_scratch_doubles(smax, 2 * d.kk)) + up32(8) + (learned ? up32(ov) : 0);
    const size_t pm = (size_t)d.pmax, n = (size_t)d.n, nv = n * d.v;
    off_prod[q] = nprod;
    nprod += (sizeof(T) == 4 ? up32(pm * ov) : 0) + up32(pm * nv) * (rpa ? 3 : 2) + up32(pm * n * n) * (rpa ? 3 : 2) +
             up32((size_t)d.np * pm) * 2;
    off_slot[q] = nslot;
    nslot += up32(mn);
    // guess: unit vectors on the lowest orbital-energy gaps
    std::vector<double> eps(m.n);
    XS_CUDA(cudaMemcpyAsync(eps.data(), m.eps.get(), sizeof(double) * m.n, cudaMemcpyDeviceToHost, s));
    XS_CUDA(cudaStreamSynchronize(s));
    guess[q] = lowest_gaps(eps, m.o, m.v, learned ? std::min<long long>(d.ov, kLearnedPairs) : nguess);
    gld = std::max(gld, nguess);
  }
  bw.dsub.ensure(nsub);
  if (sizeof(T) == 4) bw.fprod.ensure(nprod); else bw.dprod.ensure(nprod);
  bw.islot.ensure(nslot);
  for (int q = 0; q < count; ++q) {
    DevMol& m = c.mols[first + q];
    BMol& d = h[q];
    const size_t ov = (size_t)d.ov, S = (size_t)d.Smax, k2 = 2 * (size_t)d.kk, mn = (size_t)d.maxnew;
    double* p = bw.dsub.get() + off_sub[q];
    auto take = [&](size_t cnt) { double* r = p; p += up32(cnt); return r; };
    d.V = take(S * ov); d.S1 = take(S * ov); d.S2 = rpa ? take(S * ov) : nullptr;
    d.Xb = take(k2 * ov); d.Rb = rpa ? take(k2 * ov) : nullptr;
    d.T = take(mn * ov);
    d.C = take((rpa ? 3 : 2) * k2 * ov);
    d.a1 = take(S * S); d.a2 = take(S * S); d.Mb = take(S * S); d.Lb = take(S * S); d.Pb = take(S * S);
    d.Nb = take(S * S);
    d.Q = take(S * k2); d.E = take(S * k2); d.coef = take(4 * S * k2);
    d.tS = take(S * mn); d.G2 = take(mn * mn); d.Bm = take(mn * mn);
    d.wts = take(S); d.omega = take(d.kk); d.osc = take(d.kk); d.nrm = take(k2); d.tn = take(mn);
    d.dm = take(3 * (size_t)d.kk); d.gpart = take((size_t)d.nch * 2 * 4096);
    d.syw = take(syevk_scratch_doubles(d.Smax, 2 * d.kk));
    d.rhist = take(8);
    d.shift = learned ? take(ov) : nullptr;
    T* pp = (sizeof(T) == 4 ? reinterpret_cast<T*>(bw.fprod.get()) : reinterpret_cast<T*>(bw.dprod.get())) + off_prod[q];
    auto takep = [&](size_t cnt) { T* r = pp; pp += up32(cnt); return r; };
    const size_t pm = (size_t)d.pmax, n = (size_t)d.n, nv = n * d.v;
    d.Xf = sizeof(T) == 4 ? takep(pm * ov) : nullptr;
    d.Tm = takep(pm * nv); d.Sb = takep(pm * nv); d.Sq = rpa ? takep(pm * nv) : nullptr;
    d.Rm = takep(pm * n * n); d.Gp = takep(pm * n * n); d.Gq = rpa ? takep(pm * n * n) : nullptr;
    d.r = takep((size_t)d.np * pm); d.J2 = takep((size_t)d.np * pm);
    d.slot = bw.islot.get() + off_slot[q];
    d.gp_pairs = reinterpret_cast<const int2*>(m.gp_pairs.get());
    d.gp_sa = reinterpret_cast<const int4*>(m.gp_sa.get());
    d.gp_npairs = m.gp_npairs;
    d.gb_rows = reinterpret_cast<const int4*>(m.gb_rows.get());
    d.gb_cols = reinterpret_cast<const int4*>(m.gb_cols.get());
    d.ao_atom = m.ao_atom.get(); d.ao_local = m.ao_local.get(); d.atom_ao_off = m.atom_ao_off.get();
    d.atom_nao = m.atom_nao.get(); d.atom_prod_off = m.atom_prod_off.get(); d.atom_elem = m.atom_elem.get();
    d.eps = m.eps.get();
    d.dip = triplet ? nullptr : m.dip.get();
    d.CT = sizeof(T) == 4 ? static_cast<const void*>(m.CTf.get()) : static_cast<const void*>(m.CT.get());
    d.W = sizeof(T) == 4 ? static_cast<const void*>(m.Wf.get()) : static_cast<const void*>(m.W.get());
    m.nroots = d.kk;
    m.method = opt.method;
    m.spin = opt.spin;
    m.U.alloc((size_t)d.kk * ov);
    m.Wv.alloc((size_t)d.kk * ov);
    d.U = m.U.get();
    d.Wv = m.Wv.get();
  }
  for (int q = 0; q < count; ++q) cfg.smax = std::max(cfg.smax, h[q].Smax);
  bw.dmols.ensure(count);
  XS_CUDA(cudaMemcpyAsync(bw.dmols.get(), h.data(), sizeof(BMol) * count, cudaMemcpyHostToDevice, s));
  std::vector<int> hst((size_t)count * kSt, 0);
  std::vector<long long> hg((size_t)count * gld, 0);
  for (int q = 0; q < count; ++q) {
    const int ng = static_cast<int>(std::min<long long>(
        guess[q].size(), std::min<long long>(h[q].ov, std::max(2 * h[q].kk, h[q].kk + 2))));
    hst[q * kSt + F_S] = ng;
    hst[q * kSt + F_SOLD] = 0;
    hst[q * kSt + F_NNEW] = ng;
    hst[q * kSt + F_PROD] = ng;
    hst[q * kSt + F_STATUS] = BS_ACTIVE;
    for (int j = 0; j < ng; ++j) hg[(size_t)q * gld + j] = guess[q][j];
  }
  bw.dst.ensure(hst.size());
  XS_CUDA(cudaMemcpyAsync(bw.dst.get(), hst.data(), sizeof(int) * hst.size(), cudaMemcpyHostToDevice, s));
  bw.gidx.ensure(hg.size());
  XS_CUDA(cudaMemcpyAsync(bw.gidx.get(), hg.data(), sizeof(long long) * hg.size(), cudaMemcpyHostToDevice, s));
  bw.nact.ensure(1);
  if (!bw.hnact) XS_CUDA(cudaMallocHost(&bw.hnact, sizeof(int)));
  const BMol* dm = bw.dmols.get();
  int* dst = bw.dst.get();
  if (learned) {
    // features of every molecule's lowest-gap pairs, one network pass over all
    // of them (in row chunks), then per molecule the guess pairs of highest
    // predicted weight and the predicted diagonal shift on the scored pairs
    HostScope h_learned("host:learned_guess");
    std::vector<int> row0(count), nrow(count);
    int total = 0;
    for (int q = 0; q < count; ++q) {
      row0[q] = total;
      nrow[q] = static_cast<int>(guess[q].size());
      total += nrow[q];
    }
    bw.F.ensure((size_t)total * kMlpFeatures);
    bw.out.ensure((size_t)total * kMlpOutputs);
    std::vector<long long> allp((size_t)total);
    for (int q = 0; q < count; ++q) {
      std::copy(guess[q].begin(), guess[q].end(), allp.begin() + row0[q]);
      pair_features(c, c.mols[first + q], guess[q], bw.F.get() + (size_t)row0[q] * kMlpFeatures, bw.dpairs, bw.fw);
    }
    for (int r = 0; r < total; r += kForwardRows) {
      const int rows = std::min(kForwardRows, total - r);
      c.mlp->forward(s, rows, bw.F.get() + (size_t)r * kMlpFeatures, bw.Z, bw.H, bw.mo);
      XS_CUDA(cudaMemcpyAsync(bw.out.get() + (size_t)r * kMlpOutputs, bw.H[kMlpLayers - 1].get(),
                              sizeof(float) * rows * kMlpOutputs, cudaMemcpyDeviceToDevice, s));
    }
    Mlp::check(s, bw.mo);
    bw.lpairs.ensure(allp.size());
    XS_CUDA(cudaMemcpyAsync(bw.lpairs.get(), allp.data(), sizeof(long long) * allp.size(), cudaMemcpyHostToDevice, s));
    bw.lrow.ensure(2 * (size_t)count);
    std::vector<int> rr(row0);
    rr.insert(rr.end(), nrow.begin(), nrow.end());
    XS_CUDA(cudaMemcpyAsync(bw.lrow.get(), rr.data(), sizeof(int) * rr.size(), cudaMemcpyHostToDevice, s));
    for (int q = 0; q < count; ++q) XS_CUDA(cudaMemsetAsync(h[q].shift, 0, sizeof(double) * h[q].ov, s));
    bselect_kernel<<<count, 256, 0, s>>>(dm, dst, cfg, bw.lpairs.get(), bw.lrow.get(), bw.lrow.get() + count,
                                         bw.out.get(), bw.gidx.get(), gld);
    XS_CHECK_LAUNCH();
    bshift_kernel<<<kGridCTAs, 256, 0, s>>>(dm, dst, cfg, bw.lpairs.get(), bw.lrow.get(), bw.lrow.get() + count,
                                            bw.out.get());
    XS_CHECK_LAUNCH();
    XS_CUDA(cudaStreamSynchronize(s));   // the host pair lists are released after this scope
  }
  bguess_kernel<<<kGridCTAs, 256, 0, s>>>(dm, dst, cfg, bw.gidx.get(), gld);
  XS_CHECK_LAUNCH();
  set_attributes();

  // one captured graph per iteration, replayed until no molecule is active
  GraphGuard gg;
  const int per_iter = capture_mode<T>(s, dm, dst, cfg, c.d_par.get(), bw.nact.get(), bw.hnact, gg);
  int it = 0;
  for (; it <= cfg.max_iter; ++it) {
    XS_CUDA(cudaGraphLaunch(gg.e, s));
    {
      HostScope h_wait("host:fetch_wait");
      XS_CUDA(cudaStreamSynchronize(s));
    }
    if (g_prof && g_prof->on) g_prof->launches += per_iter;
    if (graph_launches) ++*graph_launches;
    if (*bw.hnact == 0) break;
  }

  // oscillator strengths, results, amplitudes
  if (!triplet) {
    bgram_kernel<GR_OSC><<<kGridCTAs, 256, 0, s>>>(dm, dst, cfg);
    XS_CHECK_LAUNCH();
    bgram_reduce_kernel<GR_OSC><<<kGridCTAs, 256, 0, s>>>(dm, dst, cfg);
    XS_CHECK_LAUNCH();
  }
  bosc_kernel<<<count, 32, 0, s>>>(dm, dst, cfg);
  XS_CHECK_LAUNCH();
  const int ldo = 3 * kBatchMaxRoots;
  bw.results.ensure((size_t)count * ldo);
  bresults_kernel<<<count, 32, 0, s>>>(dm, dst, cfg, bw.results.get(), ldo);
  XS_CHECK_LAUNCH();
  bkeep_kernel<<<kGridCTAs, 256, 0, s>>>(dm, dst, cfg);
  XS_CHECK_LAUNCH();
  std::vector<double> res((size_t)count * ldo);
  XS_CUDA(cudaMemcpyAsync(res.data(), bw.results.get(), sizeof(double) * res.size(), cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaMemcpyAsync(hst.data(), dst, sizeof(int) * hst.size(), cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < count; ++q) {
    DevMol& m = c.mols[first + q];
    const BMol& d = h[q];
    const int* sq = hst.data() + (size_t)q * kSt;
    SolveStats& ss = st[first + q];
    ss.iterations = sq[F_ITER];
    ss.products = sq[F_PROD];
    ss.converged = sq[F_STATUS] == BS_CONVERGED;
    ss.smax = d.Smax;
    ss.tol_used = cfg.tol;
    ss.learned = learned;
    ss.fallback = sq[F_NOSHIFT] != 0;
    const double* r = res.data() + (size_t)q * ldo;
    m.omega.assign(r, r + d.kk);
    m.resid.assign(r + d.kk, r + 2 * d.kk);
    m.osc.assign(r + 2 * d.kk, r + 3 * d.kk);
    m.iterations = ss.iterations;
    int rc = XS_OK;
    if (sq[F_STATUS] == BS_UNSTABLE) rc = XS_EUNSTABLE;
    else if (sq[F_STATUS] != BS_CONVERGED) rc = XS_ENOCONV;
    rcs[first + q] = rc;
  }
}

}  // namespace

void davidson_batched(Ctx& c, const xs_ex_opts& opt, std::vector<SolveStats>& st, std::vector<int>& rcs,
                      long long* graph_launches) {
  if (opt.nroots > kBatchMaxRoots)
    throw Error(XS_EINVAL, "batched solves take at most 16 roots (xs_ex_opts.batched = 2 runs molecules concurrently)");
  const int nmol = static_cast<int>(c.mols.size());
  st.assign(nmol, SolveStats{});
  rcs.assign(nmol, XS_OK);
  if (!c.batch_cache)
    c.batch_cache = std::shared_ptr<void>(new BatchWork(), [](void* p) { delete static_cast<BatchWork*>(p); });
  BatchWork& bw = *static_cast<BatchWork*>(c.batch_cache.get());
  for (int first = 0; first < nmol; first += kBatchGroup) {
    const int count = std::min(kBatchGroup, nmol - first);
    if (opt.precision == XS_MIXED) solve_group<float>(c, bw, opt, first, count, st, rcs, graph_launches);
    else solve_group<double>(c, bw, opt, first, count, st, rcs, graph_launches);
  }
}

}  // namespace xs
