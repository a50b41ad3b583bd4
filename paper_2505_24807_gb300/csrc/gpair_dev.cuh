// Device bodies of libxs's float32 G build over super-atom pairs (the
// algorithm is described at the top of gpair.cu).  Included by gpair.cu (one
// molecule per launch) and batch.cu (all molecules of a batch per launch).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gbuild_dev.cuh"
#include "kernels.h"

namespace xs {
namespace {

// super-atom: x = first AO, y = AO count (+16 for a heavy atom), z = first
// on-atom product, w = element row
__device__ __forceinline__ bool sa_heavy(int4 a) { return a.y & 16; }
__device__ __forceinline__ int sa_nao(int4 a) { return a.y & 15; }

// TF32 pair: hi and lo = x - hi both rounded to nearest TF32 (the tensor
// cores would truncate lo's low bits, a bias toward zero)
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  const uint32_t bits = __float_as_uint(x);
  hi = __uint_as_float((bits + 0x1000u) & 0xFFFFE000u);
  lo = __uint_as_float((__float_as_uint(x - hi) + 0x1000u) & 0xFFFFE000u);
}

struct PairOut {
  float *G, *Gm;                 // plain outputs (row stride n)
  float *Gh, *Gl, *Gmh, *Gml;    // TF32 pairs (row stride ldo)
  int ldo;
};

template <bool SPLIT, bool RPA>
__device__ __forceinline__ void put(const PairOut& o, int n, long long vb, int row, int col, float g, float gm) {
  if (SPLIT) {
    const long long at = vb * o.ldo + (long long)row * o.ldo + col;
    float h, l;
    tf32_split(g, h, l);
    o.Gh[at] = h;
    o.Gl[at] = l;
    if (RPA) {
      tf32_split(gm, h, l);
      o.Gmh[at] = h;
      o.Gml[at] = l;
    }
  } else {
    const long long at = vb * n + (long long)row * n + col;
    o.G[at] = g;
    if (RPA) o.Gm[at] = gm;
  }
}

// (lo, hi) AO indices of on-atom product p (s, px, py, pz; the pidx order)
__device__ __forceinline__ int plo(int p) { return p < 4 ? 0 : (p < 7 ? 1 : (p < 9 ? 2 : 3)); }
__device__ __forceinline__ int phi(int p) { return p < 4 ? p : (p < 7 ? p - 3 : (p < 9 ? p - 5 : 3)); }

// Exchange blocks of one off-diagonal pair and one matrix.  ws holds the
// pair's integrals (row stride ldw); each unique integral is read once and
// applied to every (mu nu), (lam sig) index order it stands for.
template <bool HI, bool HJ>
__device__ __forceinline__ void exchange(const float* ws, int ldw, const float (&Rij)[4][4], const float (&Rji)[4][4],
                                         float (&Kij)[4][4], float (&Kji)[4][4]) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int lam = 0; lam < 4; ++lam) {
      Kij[mu][lam] = 0.0f;
      Kji[lam][mu] = 0.0f;
    }
#pragma unroll
  for (int a = 0; a < (HI ? 10 : 4); ++a) {
    const int m0 = HI ? plo(a) : a, n0 = HI ? phi(a) : a;
#pragma unroll
    for (int b = 0; b < (HJ ? 10 : 4); ++b) {
      const int l0 = HJ ? plo(b) : b, s0 = HJ ? phi(b) : b;
      const float w = ws[a * ldw + b];
#pragma unroll
      for (int ca = 0; ca < 2; ++ca) {
        if (ca == 1 && m0 == n0) continue;
        const int mu = ca ? n0 : m0, nu = ca ? m0 : n0;
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
          if (cb == 1 && l0 == s0) continue;
          const int lam = cb ? s0 : l0, sg = cb ? l0 : s0;
          Kij[mu][lam] = fmaf(w, Rij[nu][sg], Kij[mu][lam]);
          Kji[lam][mu] = fmaf(w, Rji[sg][nu], Kji[lam][mu]);
        }
      }
    }
  }
}

// four consecutive floats of row `row` from column `col` (zero past cnt),
// one 16-byte load when aligned
__device__ __forceinline__ void load4(const float* __restrict__ base, long long ld, int row, int col, int cnt, bool vec,
                                      float (&out)[4]) {
  const float* p = base + (long long)row * ld + col;
  if (vec) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = x.x; out[1] = x.y; out[2] = x.z; out[3] = x.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = j < cnt ? __ldg(p + j) : 0.0f;
  }
}

__device__ __forceinline__ void store4(float* base, long long ld, int row, int col, int cnt, bool vec,
                                       const float (&v)[4]) {
  float* p = base + (long long)row * ld + col;
  if (vec) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < cnt) p[j] = v[j];
  }
}

// one output row segment (4 values): plain into A, or its TF32 pair into
// A (hi) and B (lo)
template <bool SPLIT>
__device__ __forceinline__ void put_row(float* A, float* B, float* unused, long long ld, int row, int col, int cnt,
                                        bool vec, const float (&g)[4]) {
  (void)unused;
  if (SPLIT) {
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tf32_split(g[j], h[j], l[j]);
    store4(A, ld, row, col, cnt, vec, h);
    store4(B, ld, row, col, cnt, vec, l);
  } else {
    store4(A, ld, row, col, cnt, vec, g);
  }
}

template <GMode MODE, bool SPLIT, bool HI, bool HJ>
__device__ __forceinline__ void offdiag_pair(int n, int nvec, int4 I, int4 J, const float* __restrict__ R,
                                             const PairOut& o, const float* ws, int ldw) {
  constexpr bool kRpa = MODE == G_RPA || MODE == G_RPA_T;
  const int nI = sa_nao(I), nJ = sa_nao(J);
  const int ldo = SPLIT ? o.ldo : n;
  // 16-byte row segments: the block starts on a multiple of 4 AOs, is 4 wide
  // and the row strides are multiples of 4
  const bool vin_ij = (n % 4 == 0) && (J.x % 4 == 0) && nJ == 4;
  const bool vin_ji = (n % 4 == 0) && (I.x % 4 == 0) && nI == 4;
  const bool vout_ij = (ldo % 4 == 0) && (J.x % 4 == 0) && nJ == 4;
  const bool vout_ji = (ldo % 4 == 0) && (I.x % 4 == 0) && nI == 4;
  // element offsets inside one matrix (32-bit: n * ld < 2^31)
  const int in_ij = I.x * n + J.x, in_ji = J.x * n + I.x;
  const int out_ij = I.x * ldo + J.x, out_ji = J.x * ldo + I.x;
  const int nn = n * n, no = n * ldo;
  float* G0 = SPLIT ? o.Gh : o.G;
  float* G1 = SPLIT ? o.Gl : nullptr;
  float* M0 = SPLIT ? o.Gmh : o.Gm;
  float* M1 = SPLIT ? o.Gml : nullptr;
  float cij[4][4], cji[4][4];
  auto fetch = [&](int v, float (&xij)[4][4], float (&xji)[4][4]) {
    const float* Rv = R + (size_t)v * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < nI) load4(Rv + in_ij, n, i, 0, nJ, vin_ij, xij[i]);
      else xij[i][0] = xij[i][1] = xij[i][2] = xij[i][3] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < nJ) load4(Rv + in_ji, n, j, 0, nI, vin_ji, xji[j]);
      else xji[j][0] = xji[j][1] = xji[j][2] = xji[j][3] = 0.0f;
    }
  };
  fetch(0, cij, cji);
  for (int v = 0; v < nvec; ++v) {
    // the next matrix's blocks are in flight while this one is contracted
    float nij[4][4], nji[4][4];
    if (v + 1 < nvec) fetch(v + 1, nij, nji);
    float Kij[4][4], Kji[4][4];
    exchange<HI, HJ>(ws, ldw, cij, cji, Kij, Kji);
    const size_t vb = (size_t)v * no;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      if (mu >= nI) continue;
      float g[4], q[4];
#pragma unroll
      for (int lam = 0; lam < 4; ++lam) {
        g[lam] = kRpa ? -(Kij[mu][lam] + Kji[lam][mu]) : -Kij[mu][lam];
        q[lam] = -(Kij[mu][lam] - Kji[lam][mu]);
      }
      put_row<SPLIT>(G0 + vb + out_ij, G1 + vb + out_ij, G1 ? G1 + vb + out_ij : nullptr, ldo, mu, 0, nJ, vout_ij, g);
      if (kRpa) put_row<SPLIT>(M0 + vb + out_ij, M1 ? M1 + vb + out_ij : nullptr, M1 ? M1 + vb + out_ij : nullptr,
                               ldo, mu, 0, nJ, vout_ij, q);
    }
#pragma unroll
    for (int lam = 0; lam < 4; ++lam) {
      if (lam >= nJ) continue;
      float g[4], q[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        g[mu] = kRpa ? -(Kij[mu][lam] + Kji[lam][mu]) : -Kji[lam][mu];
        q[mu] = Kij[mu][lam] - Kji[lam][mu];
      }
      put_row<SPLIT>(G0 + vb + out_ji, G1 ? G1 + vb + out_ji : nullptr, G1 ? G1 + vb + out_ji : nullptr, ldo, lam, 0,
                     nI, vout_ji, g);
      if (kRpa) put_row<SPLIT>(M0 + vb + out_ji, M1 ? M1 + vb + out_ji : nullptr, M1 ? M1 + vb + out_ji : nullptr,
                               ldo, lam, 0, nI, vout_ji, q);
    }
    if (v + 1 < nvec) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cij[i][j] = nij[i][j];
          cji[i][j] = nji[i][j];
        }
    }
  }
}

// diagonal block of a super-atom: one-centre Coulomb and exchange, the
// two-centre Coulomb of the diagonal blocks (J2), and for a hydrogen run the
// exchange between its hydrogens
template <GMode MODE, bool SPLIT>
__device__ __forceinline__ void diag_block(int n, int np, int nvec, int4 I, const double* __restrict__ par,
                                           const float* __restrict__ W, const float* __restrict__ J2, int ldj,
                                           const float* __restrict__ R, const PairOut& o) {
  constexpr bool kRpa = MODE == G_RPA || MODE == G_RPA_T;
  constexpr bool kTriplet = MODE == G_CIS_T || MODE == G_RPA_T;
  const long long nn = (long long)n * n;
  const double* pd = par + I.w * XS_NPARAM;
  if (sa_heavy(I)) {
    float p[XS_NPARAM];
#pragma unroll
    for (int i = 0; i < XS_NPARAM; ++i) p[i] = (i >= 4 && i <= 8) ? static_cast<float>(pd[i]) : 0.0f;
    for (int v = 0; v < nvec; ++v) {
      float Rd[16];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Rd[i * 4 + j] = R[v * nn + (long long)(I.x + i) * n + I.x + j];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float J1, K1ab, K1ba;
          one_centre<float>(p, a, b, Rd, J1, K1ab, K1ba);
          float g, gm = 0.0f;
          if (kTriplet) {
            g = kRpa ? -(K1ab + K1ba) : -K1ab;
            if (kRpa) gm = -(K1ab - K1ba);
          } else {
            const float J = J1 + J2[(long long)(I.z + pidx(a, b)) * ldj + v];
            if (!kRpa) {
              g = 2.0f * J - K1ab;
            } else {
              g = 4.0f * J - (K1ab + K1ba);
              gm = -(K1ab - K1ba);
            }
          }
          put<SPLIT, kRpa>(o, n, v * (long long)n, I.x + a, I.x + b, g, gm);
        }
    }
    return;
  }
  const int nI = sa_nao(I);
  const float gss = static_cast<float>(pd[4]);
  float w[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = (i < nI && j < nI && i != j) ? W[(long long)(I.z + i) * np + I.z + j] : 0.0f;
  for (int v = 0; v < nvec; ++v) {
    float Rd[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        Rd[i][j] = (i < nI && j < nI) ? R[v * nn + (long long)(I.x + i) * n + I.x + j] : 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (i >= nI || j >= nI) continue;
        float g, gm = 0.0f;
        if (i == j) {
          const float k1 = gss * Rd[i][i];
          if (kTriplet) {
            g = kRpa ? -2.0f * k1 : -k1;
          } else {
            const float J = k1 + J2[(long long)(I.z + i) * ldj + v];
            g = kRpa ? 4.0f * J - 2.0f * k1 : 2.0f * J - k1;
          }
        } else {
          const float kr = w[i][j] * Rd[i][j], krt = w[i][j] * Rd[j][i];
          g = kRpa ? -(kr + krt) : -kr;
          gm = -(kr - krt);
        }
        put<SPLIT, kRpa>(o, n, v * (long long)n, I.x + i, I.x + j, g, gm);
      }
  }
}

// One super-atom pair of the pair list, all nvec matrices; ws: 100 floats of
// shared memory owned by the calling thread.
template <GMode MODE, bool SPLIT>
__device__ __forceinline__ void gpair_one(int n, int np, int nvec, int2 pr, const int4* __restrict__ sa,
                                          const double* __restrict__ par, const float* __restrict__ W,
                                          const float* __restrict__ J2, int ldj, const float* __restrict__ R,
                                          const PairOut& o, float* ws) {
  if (pr.x < 0) return;
  const int4 I = sa[pr.x];
  if (pr.x == pr.y) {
    diag_block<MODE, SPLIT>(n, np, nvec, I, par, W, J2, ldj, R, o);
    return;
  }
  const int4 J = sa[pr.y];
  const bool hI = sa_heavy(I), hJ = sa_heavy(J);
  const int npI = hI ? 10 : sa_nao(I), npJ = hJ ? 10 : sa_nao(J);
  for (int a = 0; a < (hI ? 10 : 4); ++a)
    for (int b = 0; b < (hJ ? 10 : 4); ++b)
      ws[a * 10 + b] = (a < npI && b < npJ) ? __ldg(W + (long long)(I.z + a) * np + J.z + b) : 0.0f;
  const int kind = (hI ? 2 : 0) + (hJ ? 1 : 0);
  switch (kind) {
    case 3: offdiag_pair<MODE, SPLIT, true, true>(n, nvec, I, J, R, o, ws, 10); break;
    case 2: offdiag_pair<MODE, SPLIT, true, false>(n, nvec, I, J, R, o, ws, 10); break;
    case 1: offdiag_pair<MODE, SPLIT, false, true>(n, nvec, I, J, R, o, ws, 10); break;
    default: offdiag_pair<MODE, SPLIT, false, false>(n, nvec, I, J, R, o, ws, 10); break;
  }
}

}  // namespace
}  // namespace xs
