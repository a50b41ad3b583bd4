// G(R) build of libxs: the NDDO two-electron contraction of the A*X product.
//
// Paper, Section "GPU Implementation", Eq. ftilde:
//   Ft_{mu nu} = sum_{lam sig} [(mu nu|lam sig) - (mu lam|nu sig)] R_{lam sig},
// with NDDO leaving Coulomb on the diagonal atom blocks (symmetrised R) and
// exchange everywhere, contracted with the symmetric and antisymmetric parts
// of R.  With J(R) = sum (mu nu|lam sig) R and K(R) = sum (mu lam|nu sig) R the
// singlet products need (spin adaptation, see xs.h):
//   CIS (and the Fock build at P = D/2):  G  = 2 J(R) - K(R)
//   TDHF:                                 G+ = 4 J(Rs) - 2 K(Rs) = 4 J(R) - K(R) - K(R^T)
//                                         G- = -2 K(Ra)          = -K(R) + K(R^T)
//
// Three steps per batch of nvec matrices:
//   1. pack the diagonal atom blocks of R into product vectors r_B[q]
//      (R_ls + R_sl for l < s, R_ll on the diagonal);
//   2. two-centre Coulomb J2 = W r with the dense product supermatrix W
//      (one GEMM over the batch: W is read once per batch);
//   3. atom-aligned tiles of G (one row group x one column tile per CTA, the
//      tile's pair-integral block staged once in shared memory, the nvec
//      matrices streamed through it): diagonal atom blocks combine J2 with the
//      closed-form one-centre Coulomb/exchange; off-diagonal blocks hold the
//      two-centre exchange sum_{nu in A, sig in B} (mu nu|lam sig) R_{nu sig}.
#include <vector>

#include "kernels.h"
#include "model.h"
#include "prof.h"
#include "gbuild_dev.cuh"

namespace xs {

namespace {

// Atom-aligned tiles of G: a CTA owns one row group (a heavy atom's 4 AOs, or
// up to 4 consecutive hydrogens) and one column tile (whole atoms, at most 64
// AOs).  It stages the pair-integral block W[products of the rows' atoms]
// [products of the columns' atoms] in shared memory once and then streams the
// nvec matrices in groups of GV: per matrix, R's tile (and for TDHF its
// transpose tile) goes through shared memory and every thread writes one G
// (and G-) element.  The next group's tiles are loaded into registers while
// the current group is computed, so each thread keeps GV loads in flight (the
// loads are 4-byte elements: one matrix at a time left HBM mostly idle).
template <typename T>
__host__ __device__ constexpr int gv_for() { return sizeof(T) == 4 ? 4 : 1; }   // float32: 4 matrices per group (shared memory)

// TF32 pair of a float (hi and lo = x - hi both rounded to nearest TF32: the
// tensor cores would otherwise truncate lo's low bits, a bias toward zero):
// the split epilogue writes the tensor-core operand of the back-transform
// directly
__device__ __forceinline__ void tf32_pair(float x, float& hi, float& lo) {
  const uint32_t bits = __float_as_uint(x);
  hi = __uint_as_float((bits + 0x1000u) & 0xFFFFE000u);
  lo = __uint_as_float((__float_as_uint(x - hi) + 0x1000u) & 0xFFFFE000u);
}

// Output of the tile kernel: plain G (and G-) with row stride n, or (SPLIT)
// their TF32 pairs with row stride ldo (batch stride n * ldo)
template <typename T>
struct GOut {
  T* G;
  T* Gm;
  float *Gh, *Gl, *Gmh, *Gml;
  int ldo;
};

template <typename T, GMode MODE, bool SPLIT>
__global__ void __launch_bounds__(256, 4) gtile_kernel(int n, int np, int nvec, const int4* __restrict__ rows,
                                                    const int4* __restrict__ cols, const int* __restrict__ ao_atom,
                                                    const int* __restrict__ ao_local,
                                                    const int* __restrict__ atom_ao_off,
                                                    const int* __restrict__ atom_nao,
                                                    const int* __restrict__ atom_prod_off,
                                                    const int* __restrict__ atom_elem,
                                                    const double* __restrict__ par, const T* __restrict__ W,
                                                    const T* __restrict__ J2, const T* __restrict__ Rall,
                                                    const GOut<T> out) {
  // R tiles padded by 4 rows / columns of zeros: a hydrogen's block is
  // handled as a 4 x 4 block with zero weights past its single AO
  // double-buffered groups: group g is read from one buffer while group g + 1
  // is stored into the other from registers loaded before the compute
  constexpr int GV = gv_for<T>();
  constexpr bool kRpa = MODE == G_RPA || MODE == G_RPA_T;       // G+ and G- outputs, R^T tiles
  constexpr bool kTriplet = MODE == G_CIS_T || MODE == G_RPA_T;  // no Coulomb terms
  __shared__ T Ws[kGP][kGQ + 1];
  __shared__ T Rt[2][GV][kGR + 4][kGC + 4];
  __shared__ T Rtt[2][GV][kGC + 4][kGR + 5];   // odd row stride: the rows of different atoms hit different banks
  const int4 rg = rows[blockIdx.y], ct = cols[blockIdx.x];
  const int ra = rg.x, nr = rg.y, cb = ct.x, nc = ct.y;
  const int PA0 = atom_prod_off[rg.z], PB0 = atom_prod_off[ct.z];
  const int nPA = atom_prod_off[rg.w - 1] + (atom_nao[rg.w - 1] == 4 ? 10 : 1) - PA0;
  const int nPB = atom_prod_off[ct.w - 1] + (atom_nao[ct.w - 1] == 4 ? 10 : 1) - PB0;
  const int tid = threadIdx.x;
  // one warp per pair-integral row, lanes along the row (no integer division)
  for (int pr = tid >> 5; pr < nPA; pr += blockDim.x >> 5)
    for (int pc = tid & 31; pc < nPB; pc += 32) Ws[pr][pc] = W[(long long)(PA0 + pr) * np + PB0 + pc];
  for (int idx = tid; idx < 2 * GV * (kGR + 4) * (kGC + 4); idx += blockDim.x) (&Rt[0][0][0][0])[idx] = T(0);
  for (int idx = tid; idx < 2 * GV * (kGC + 4) * (kGR + 5); idx += blockDim.x) (&Rtt[0][0][0][0])[idx] = T(0);
  const int ri = tid / kGC, ci = tid % kGC;
  const bool active = ri < nr && ci < nc;
  const int mu = ra + ri, lam = cb + ci;
  int A = 0, B = 0, a = 0, b = 0, nA = 1, nB = 1, rA = 0, cA = 0, rB = 0, pA = 0, pB = 0, PA = 0;
  const double* pd = par;   // the diagonal block's element parameters (read where used)
  if (active) {
    A = ao_atom[mu]; B = ao_atom[lam];
    a = ao_local[mu]; b = ao_local[lam];
    nA = atom_nao[A]; nB = atom_nao[B];
    rA = atom_ao_off[A] - ra;          // A's first row in the tile
    cA = atom_ao_off[A] - cb;          // A's first column (diagonal block)
    rB = atom_ao_off[B] - cb;          // B's first column in the tile
    PA = atom_prod_off[A];
    pA = PA - PA0;
    pB = atom_prod_off[B] - PB0;
    if (A == B) pd = par + atom_elem[A] * XS_NPARAM;
  }
  __syncthreads();
  // this output's 16 exchange weights (mu nu|lam sig) for nu in A, sig in B,
  // zero past a hydrogen's single AO; independent of the matrix index
  T wv[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) wv[q] = T(0);
  if (active && A != B) {
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
#pragma unroll
      for (int sg = 0; sg < 4; ++sg)
        if (nu < nA && sg < nB)
          wv[nu * 4 + sg] = Ws[pA + ((nA == 4) ? pidx(a, nu) : 0)][pB + ((nB == 4) ? pidx(b, sg) : 0)];
  }
  const int tr = tid % kGR, tc = tid / kGR;   // transpose tile: 4 consecutive threads per row
  const bool tact = kRpa && tr < nr && tc < nc;
  const long long nn = (long long)n * n;
  const long long at_r = (long long)mu * n + lam, at_t = (long long)(cb + tc) * n + ra + tr;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < GV; ++q) {
    if (q < nvec) {
      if (active) Rt[0][q][ri][ci] = Rall[q * nn + at_r];
      if (tact) Rtt[0][q][tc][tr] = Rall[q * nn + at_t];
    }
  }
  __syncthreads();
  int buf = 0;
  for (int v0 = 0; v0 < nvec; v0 += GV) {
    // prefetch the next group into registers
    T nxt[GV], nxtt[GV];
#pragma unroll
    for (int q = 0; q < GV; ++q) {
      nxt[q] = T(0);
      nxtt[q] = T(0);
      const int vn = v0 + GV + q;
      if (vn < nvec) {
        if (active) nxt[q] = Rall[vn * nn + at_r];
        if (tact) nxtt[q] = Rall[vn * nn + at_t];
      }
    }
#pragma unroll
    for (int q = 0; q < GV; ++q) {
      const int v = v0 + q;
      if (!active || v >= nvec) continue;
      T g, gm = T(0);
      if (A == B) {
        T J1, K1ab, K1ba;
        if (nA == 1) {
          const T r00 = Rt[buf][q][rA][cA];
          const T gss = T(pd[4]);
          J1 = gss * r00;
          K1ab = K1ba = gss * r00;
        } else {
          T Rd[16];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Rd[i * 4 + j] = Rt[buf][q][rA + i][cA + j];
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
          const T J = J1 + J2[(long long)(PA + pab) * nvec + v];
          if (!kRpa) {
            g = T(2) * J - K1ab;
          } else {
            g = T(4) * J - (K1ab + K1ba);
            gm = -(K1ab - K1ba);
          }
        }
      } else {
        // K(R)_{mu lam} = sum_{nu in A, sig in B} (mu nu|lam sig) R_{nu sig},
        // K(R^T)_{mu lam} = sum (mu nu|lam sig) R_{sig nu}; a hydrogen has
        // one AO, so only the nonzero weights are visited (warps are nearly
        // always uniform in the atom kinds: heavy atoms precede hydrogens in
        // the AO order of the generated molecules).  The terms come in the
        // same order as in the full 4 x 4 sum, so the result is identical.
        T kr = T(0), krt = T(0);
        if (nA == 4 && nB == 4) {
#pragma unroll
          for (int nu = 0; nu < 4; ++nu)
#pragma unroll
            for (int sg = 0; sg < 4; ++sg) {
              kr = fma(wv[nu * 4 + sg], Rt[buf][q][rA + nu][rB + sg], kr);
              if (kRpa) krt = fma(wv[nu * 4 + sg], Rtt[buf][q][rB + sg][rA + nu], krt);
            }
        } else if (nA == 4) {
#pragma unroll
          for (int nu = 0; nu < 4; ++nu) {
            kr = fma(wv[nu * 4], Rt[buf][q][rA + nu][rB], kr);
            if (kRpa) krt = fma(wv[nu * 4], Rtt[buf][q][rB][rA + nu], krt);
          }
        } else if (nB == 4) {
#pragma unroll
          for (int sg = 0; sg < 4; ++sg) {
            kr = fma(wv[sg], Rt[buf][q][rA][rB + sg], kr);
            if (kRpa) krt = fma(wv[sg], Rtt[buf][q][rB + sg][rA], krt);
          }
        } else {
          kr = fma(wv[0], Rt[buf][q][rA][rB], kr);
          if (kRpa) krt = fma(wv[0], Rtt[buf][q][rB][rA], krt);
        }
        if (!kRpa) {
          g = -kr;
        } else {
          g = -(kr + krt);
          gm = -(kr - krt);
        }
      }
      if constexpr (SPLIT) {
        const long long at = (long long)v * n * out.ldo + (long long)mu * out.ldo + lam;
        float h, l;
        tf32_pair(static_cast<float>(g), h, l);
        out.Gh[at] = h;
        out.Gl[at] = l;
        if (kRpa) {
          tf32_pair(static_cast<float>(gm), h, l);
          out.Gmh[at] = h;
          out.Gml[at] = l;
        }
      } else {
        out.G[v * nn + at_r] = g;
        if (kRpa) out.Gm[v * nn + at_r] = gm;
      }
    }
    if (v0 + GV < nvec) {
#pragma unroll
      for (int q = 0; q < GV; ++q) {
        if (active) Rt[buf ^ 1][q][ri][ci] = nxt[q];
        if (tact) Rtt[buf ^ 1][q][tc][tr] = nxtt[q];
      }
    }
    __syncthreads();
    buf ^= 1;
  }
}

template <typename T, GMode MODE, bool SPLIT>
void launch_mode(cudaStream_t s, const DevMol& m, const double* d_par, int nvec, const T* W, const T* J2, const T* R,
                 const GOut<T>& out) {
  dim3 grid(m.gb_ncols, m.gb_nrows);
  const int4* rows = reinterpret_cast<const int4*>(m.gb_rows.get());
  const int4* cols = reinterpret_cast<const int4*>(m.gb_cols.get());
  gtile_kernel<T, MODE, SPLIT><<<grid, 256, 0, s>>>(m.n, m.np, nvec, rows, cols, m.ao_atom.get(), m.ao_local.get(),
                                                    m.atom_ao_off.get(), m.atom_nao.get(), m.atom_prod_off.get(),
                                                    m.atom_elem.get(), d_par, W, J2, R, out);
}

template <typename T, bool SPLIT>
void launch_tiles(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const T* W, const T* J2,
                  const T* R, const GOut<T>& out) {
  switch (mode) {
    case G_CIS: launch_mode<T, G_CIS, SPLIT>(s, m, d_par, nvec, W, J2, R, out); break;
    case G_RPA: launch_mode<T, G_RPA, SPLIT>(s, m, d_par, nvec, W, J2, R, out); break;
    case G_CIS_T: launch_mode<T, G_CIS_T, SPLIT>(s, m, d_par, nvec, W, J2, R, out); break;
    case G_RPA_T: launch_mode<T, G_RPA_T, SPLIT>(s, m, d_par, nvec, W, J2, R, out); break;
  }
  XS_CHECK_LAUNCH();
}

inline bool has_coulomb(GMode mode) { return mode == G_CIS || mode == G_RPA; }
inline bool has_minus(GMode mode) { return mode == G_RPA || mode == G_RPA_T; }

// zero columns [n, ldo) of rows x ldo matrices (batch stride rows * ldo)
__global__ void zero_pad_cols_kernel(int rows, int n, int ldo, int nvec, float* a, float* b) {
  const int w = ldo - n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nvec * rows * w) return;
  const long long r = idx / w;
  const long long at = r * ldo + n + idx % w;
  a[at] = 0.0f;
  if (b) b[at] = 0.0f;
}

}  // namespace

template <typename T>
void gbuild(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const T* R, T* G, T* Gm,
            DevBuf<T>& ws) {
  if (nvec <= 0) return;
  const int n = m.n, np = m.np;
  ws.ensure((size_t)2 * np * nvec);
  T* rT = ws.get();
  T* J2 = ws.get() + (size_t)np * nvec;
  const T* W = nullptr;
  if constexpr (sizeof(T) == 8) W = reinterpret_cast<const T*>(m.W.get());
  else W = reinterpret_cast<const T*>(m.Wf.get());
  if (has_coulomb(mode)) {
    dim3 block(8, 32);
    dim3 grid((m.L.natoms + 31) / 32);
    if constexpr (sizeof(T) == 4) {
      pack_diag_kernel<T, false><<<grid, block, 0, s>>>(m.L.natoms, n, np, nvec, m.atom_ao_off.get(),
                                                        m.atom_nao.get(), m.atom_prod_off.get(), R, rT);
      XS_CHECK_LAUNCH();
      static thread_local DevBuf<float> j2_ws;
      coulomb_j2(s, np, nvec, W, rT, J2, j2_ws);
    } else {
      pack_diag_kernel<T, true><<<grid, block, 0, s>>>(m.L.natoms, n, np, nvec, m.atom_ao_off.get(),
                                                       m.atom_nao.get(), m.atom_prod_off.get(), R, rT);
      XS_CHECK_LAUNCH();
      // two-centre Coulomb J2 = W r: W streamed once, split over its columns so
      // that the skinny product fills the GPU
      static thread_local DevBuf<T> split_ws;
      gram<T>(s, np, nvec, np, W, np, rT, np, J2, nvec, T(1), T(0), split_ws);
    }
  }
  // algorithmic traffic: read R, write G (and G-), read the pair integrals once
  const double outs = has_minus(mode) ? 2.0 : 1.0;
  ProfScope ps(s, sizeof(T) == 8 ? "gbuild_assemble_f64" : "gbuild_assemble_f32",
               sizeof(T) * ((double)nvec * n * n * (1.0 + outs) + (double)np * np), 0.0);
  if constexpr (sizeof(T) == 4)
    gpair_build(s, m, d_par, mode, nvec, W, J2, nvec, R, G, Gm);
  else
    launch_tiles<T, false>(s, m, d_par, mode, nvec, W, J2, R, GOut<T>{G, Gm, nullptr, nullptr, nullptr, nullptr, 0});
}

void gbuild_split(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* R,
                  float* Gh, float* Gl, float* Gmh, float* Gml, int ldo, DevBuf<float>& ws) {
  if (nvec <= 0) return;
  const int n = m.n, np = m.np;
  if (ldo < n) throw Error(XS_EINVAL, "gbuild_split: row stride below n");
  ws.ensure((size_t)2 * np * nvec);
  float* rT = ws.get();
  float* J2 = ws.get() + (size_t)np * nvec;
  const float* W = m.Wf.get();
  if (has_coulomb(mode)) {
    dim3 block(8, 32);
    dim3 grid((m.L.natoms + 31) / 32);
    pack_diag_kernel<float, false><<<grid, block, 0, s>>>(m.L.natoms, n, np, nvec, m.atom_ao_off.get(),
                                                          m.atom_nao.get(), m.atom_prod_off.get(), R, rT);
    XS_CHECK_LAUNCH();
    static thread_local DevBuf<float> j2_ws;
    coulomb_j2(s, np, nvec, W, rT, J2, j2_ws);
  }
  if (ldo > n) {
    const long long cnt = (long long)nvec * n * (ldo - n);
    zero_pad_cols_kernel<<<grid1(cnt, 256), 256, 0, s>>>(n, n, ldo, nvec, Gh, Gl);
    if (has_minus(mode)) zero_pad_cols_kernel<<<grid1(cnt, 256), 256, 0, s>>>(n, n, ldo, nvec, Gmh, Gml);
    XS_CHECK_LAUNCH();
  }
  // algorithmic traffic: read R, write the G (and G-) TF32 pairs, read the pair integrals once
  const double outs = has_minus(mode) ? 2.0 : 1.0;
  ProfScope ps(s, "gbuild_assemble_f32", 4.0 * ((double)nvec * n * n * (1.0 + 2.0 * outs) + (double)np * np), 0.0);
  gpair_build_split(s, m, d_par, mode, nvec, W, J2, nvec, R, Gh, Gl, Gmh, Gml, ldo);
}

template <typename T>
void gbuild_raw(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const T* R, T* G, T* Gm,
                T* r, T* J2) {
  if (nvec <= 0) return;
  const int n = m.n, np = m.np;
  {
    dim3 block(8, 32);
    dim3 grid((m.L.natoms + 31) / 32);
    pack_diag_kernel<T, false><<<grid, block, 0, s>>>(m.L.natoms, n, np, nvec, m.atom_ao_off.get(),
                                                      m.atom_nao.get(), m.atom_prod_off.get(), R, r);
    XS_CHECK_LAUNCH();
  }
  const T* W = nullptr;
  if constexpr (sizeof(T) == 8) W = reinterpret_cast<const T*>(m.W.get());
  else W = reinterpret_cast<const T*>(m.Wf.get());
  gemm<T>(s, false, false, np, nvec, np, T(1), W, np, 0, r, nvec, 0, T(0), J2, nvec, 0, 1);
  launch_tiles<T, false>(s, m, d_par, mode, nvec, W, J2, R, GOut<T>{G, Gm, nullptr, nullptr, nullptr, nullptr, 0});
}

void build_gtiles(cudaStream_t s, DevMol& m) {
  const MolLayout& L = m.L;
  std::vector<int> rows, cols;   // per tile: first AO, AO count, first atom, end atom
  for (int A = 0; A < L.natoms;) {
    int A1 = A, cnt = 0;
    if (L.nao_atom[A] == 4) {
      A1 = A + 1;
      cnt = 4;
    } else {
      while (A1 < L.natoms && L.nao_atom[A1] == 1 && cnt < kGR) { ++A1; ++cnt; }
    }
    rows.insert(rows.end(), {L.ao_off[A], cnt, A, A1});
    A = A1;
  }
  for (int A = 0; A < L.natoms;) {
    int A1 = A, cnt = 0;
    while (A1 < L.natoms && cnt + L.nao_atom[A1] <= kGC) { cnt += L.nao_atom[A1]; ++A1; }
    cols.insert(cols.end(), {L.ao_off[A], cnt, A, A1});
    A = A1;
  }
  m.gb_nrows = static_cast<int>(rows.size() / 4);
  m.gb_ncols = static_cast<int>(cols.size() / 4);
  m.gb_rows.alloc(rows.size());
  m.gb_cols.alloc(cols.size());
  XS_CUDA(cudaMemcpyAsync(m.gb_rows.get(), rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, s));
  XS_CUDA(cudaMemcpyAsync(m.gb_cols.get(), cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice, s));
  XS_CUDA(cudaStreamSynchronize(s));
}

template void gbuild<double>(cudaStream_t, const DevMol&, const double*, GMode, int, const double*, double*,
                             double*, DevBuf<double>&);
template void gbuild_raw<double>(cudaStream_t, const DevMol&, const double*, GMode, int, const double*, double*,
                                 double*, double*, double*);
template void gbuild<float>(cudaStream_t, const DevMol&, const double*, GMode, int, const float*, float*, float*,
                            DevBuf<float>&);

}  // namespace xs
