// Device helpers of libxs's G(R) build shared by gbuild.cu (one molecule per
// launch) and batch.cu (all molecules of a batch per launch): the on-atom
// product index, the closed-form one-centre Coulomb and exchange terms, and
// the atom-aligned tile sizes.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace xs {
namespace {

// G tiles: a row group holds one heavy atom (4 AOs) or up to 4 hydrogens; a
// column tile holds whole atoms, at most 64 AOs; the pair-integral block of a
// tile is at most 10 x 160 products.
constexpr int kGR = 4, kGC = 64, kGP = 10, kGQ = 160;

__device__ __forceinline__ int pidx(int a, int b) {
  // product index of AOs a, b (0 = s, 1..3 = p) on a heavy atom
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  // rows: s: 0 1 2 3 | x: 4 5 6 | y: 7 8 | z: 9; row lo starts at
  // lo (9 - lo) / 2 = 0, 4, 7, 9 (arithmetic: no local-memory table)
  return ((lo * (9 - lo)) >> 1) + (hi - lo);
}

// product vectors of the diagonal atom blocks: r[q][v] (TR = false) or its
// transpose r[v][q] (TR = true, the operand of the split-K product W r)
template <typename T, bool TR>
__global__ void pack_diag_kernel(int natoms, int n, int np, int nvec, const int* __restrict__ atom_ao_off,
                                 const int* __restrict__ atom_nao, const int* __restrict__ atom_prod_off,
                                 const T* __restrict__ R, T* __restrict__ r) {
  int A = blockIdx.x * blockDim.y + threadIdx.y;
  int v = threadIdx.x;
  if (A >= natoms) return;
  for (; v < nvec; v += blockDim.x) {
    const T* Rv = R + (long long)v * n * n;
    int o = atom_ao_off[A], P = atom_prod_off[A];
    auto at = [&](int q) -> T& { return TR ? r[(long long)v * np + q] : r[(long long)q * nvec + v]; };
    if (atom_nao[A] == 1) {
      at(P) = Rv[(long long)o * n + o];
    } else {
      for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b) {
          T val = Rv[(long long)(o + a) * n + o + b];
          if (b != a) val += Rv[(long long)(o + b) * n + o + a];
          at(P + pidx(a, b)) = val;
        }
    }
  }
}

// one-centre Coulomb J1 and exchange K1 of element e at AO pair (a, b) of a
// heavy atom, from the 4x4 diagonal block Rd (row-major) -- closed forms of
// the parameters gss, gsp, gpp, gp2, hsp and hpp = (gpp - gp2)/2.
template <typename T>
__device__ __forceinline__ void one_centre(const T* p, int a, int b, const T Rd[16], T& J1, T& K1ab, T& K1ba) {
  const T gss = p[4], gsp = p[5], gpp = p[6], gp2 = p[7], hsp = p[8];
  const T hpp = T(0.5) * (gpp - gp2);
  auto R = [&](int i, int j) { return Rd[i * 4 + j]; };
  auto K1 = [&](int x, int y) -> T {
    if (x == 0 && y == 0) return gss * R(0, 0) + hsp * (R(1, 1) + R(2, 2) + R(3, 3));
    if (x == 0) return gsp * R(0, y) + hsp * R(y, 0);
    if (y == 0) return gsp * R(x, 0) + hsp * R(0, x);
    if (x == y) {
      T s = T(0);
      for (int j = 1; j < 4; ++j) if (j != x) s += R(j, j);
      return hsp * R(0, 0) + gpp * R(x, x) + hpp * s;
    }
    return gp2 * R(x, y) + hpp * R(y, x);
  };
  if (a == 0 && b == 0) {
    J1 = gss * R(0, 0) + gsp * (R(1, 1) + R(2, 2) + R(3, 3));
  } else if (a == 0 || b == 0) {
    int i = a + b;
    J1 = hsp * (R(0, i) + R(i, 0));
  } else if (a == b) {
    T s = T(0);
    for (int j = 1; j < 4; ++j) if (j != a) s += R(j, j);
    J1 = gsp * R(0, 0) + gpp * R(a, a) + gp2 * s;
  } else {
    J1 = hpp * (R(a, b) + R(b, a));
  }
  K1ab = K1(a, b);
  K1ba = K1(b, a);
}

}  // namespace
}  // namespace xs
