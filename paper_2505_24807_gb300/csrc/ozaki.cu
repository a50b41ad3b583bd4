// Float64-accurate Davidson subspace products on the BF16 tensor cores
// (tcgen05 + TMA, sm_103a) by exact digit splitting (Ozaki, Ogita, Oishi and
// Rump, Numer. Algorithms 59, 95-118 (2012)); the representation is described
// in ozaki.h.
//
// One kernel, two shapes, both with K-major digit operands:
//   gram  (mode 0)  C[m][n] = sum_l A[m][l] B[n][l]: rows of the MMA are the
//                   digit planes (m, i) of A, columns the planes (n, j) of B,
//                   K = l in exact chunks of 4096; the epilogue folds the 64
//                   digit pairs with weights 2^(-7(i+j)) into a float64
//                   partial per (chunk, m, n), summed in fixed order after.
//   combine (mode 1) Y[k][l] = sum_m c[m][k] X[m][l]: rows are l, K = the
//                   digit planes (block, m, i) of the stored vectors, columns
//                   (k, t) hold the coefficient digits on the anti-diagonals
//                   t = i + j of the digit pairs, so one float32 accumulator per
//                   (l, k, t) sums exact integers; the epilogue weights t by
//                   2^(-7t) (pairs with i + j > 9 fall below float64 rounding).
// Persistent CTAs (one per SM) walk the tiles: warp 0 issues TMA loads
// through a STAGES-deep mbarrier ring that runs on across tiles, warp 1 owns
// TMEM and issues the MMAs (M = 128, N = BN, K = 16 per instruction) into two
// alternating accumulators, warps 2-5 drain one accumulator while the next
// tile accumulates in the other.  The epilogue folds the eight float32
// digit sums with integer arithmetic (horner8) and two float64 conversions:
// this part's float64 pipe is narrow.  Every wait is bounded; a timeout
// raises the error word and the CTA leaves after draining what it issued.
#include <algorithm>

#include "kernels.h"
#include "ozaki.h"
#include "prof.h"
#include "tcgen05.cuh"

namespace xs {

namespace {

using namespace tc5;

constexpr int BM = 128;
constexpr int BKE = 64;                     // bf16 per K block: one 128-byte swizzle row
constexpr int KB_CHUNK = kOzChunk / BKE;    // K blocks per exact float32 chunk

// Balanced base-128 digits of x 2^-e (|x| < 2^(e-1)): x 2^-e = sum_i d[i] 2^(-7(i+1))
// up to a rounding of 2^-57; |d[i]| <= 64.  Integer arithmetic on the IEEE
// fields: the magnitude is rounded to a 56-bit fixed-point integer q, then
// peeled into digits from the least significant end.
__device__ __forceinline__ void oz_digits(double x, int e, int* d) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int exf = static_cast<int>((bits >> 52) & 0x7FF);
#pragma unroll
  for (int i = 0; i < kOzDigits; ++i) d[i] = 0;
  if (exf == 0 || exf == 0x7FF) return;   // zero / subnormal (below 2^-1022) / non-finite (flagged elsewhere)
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  int sh = exf - 1019 - e;                 // q = mant 2^sh
  unsigned long long q;
  if (sh >= 0) {
    q = mant << (sh > 2 ? 2 : sh);
  } else {
    const int rs = -sh;
    q = rs >= 64 ? 0ull : (((mant >> (rs - 1)) + 1ull) >> 1);
  }
  const long long r = (bits >> 63) ? -static_cast<long long>(q) : static_cast<long long>(q);
  // r = hi 2^28 + lo with 0 <= lo < 2^28: four digits from lo, its carry into
  // hi, three more digits and the remainder from hi, all in 32-bit arithmetic
  int lo = static_cast<int>(r & 0xFFFFFFF);
  int hi = static_cast<int>(r >> 28);
#pragma unroll
  for (int i = kOzDigits - 1; i >= 4; --i) {
    const int di = ((lo + 64) & 127) - 64;
    d[i] = di;
    lo = (lo - di) >> 7;
  }
  hi += lo;
#pragma unroll
  for (int i = 3; i >= 1; --i) {
    const int di = ((hi + 64) & 127) - 64;
    d[i] = di;
    hi = (hi - di) >> 7;
  }
  d[0] = hi;
}

__device__ __forceinline__ uint32_t digit_bits(int d) {
  return __float_as_uint(static_cast<float>(d)) >> 16;   // exact: |d| <= 64
}

__device__ __forceinline__ uint4 pack8(const int* d) {
  uint4 u;
  u.x = digit_bits(d[0]) | (digit_bits(d[1]) << 16);
  u.y = digit_bits(d[2]) | (digit_bits(d[3]) << 16);
  u.z = digit_bits(d[4]) | (digit_bits(d[5]) << 16);
  u.w = digit_bits(d[6]) | (digit_bits(d[7]) << 16);
  return u;
}

struct OzArgs {
  int mode;          // 0: gram partials, 1: combination
  int ntiles;        // work tiles of the launch
  int n_mtiles;      // mode 0: 128-row tiles of A (tile t: row tile t % n_mtiles, chunk t / n_mtiles)
  int kb_total;      // K blocks of the whole product (mode 0)
  int kb_per_cta;    // mode 0: K blocks per chunk; mode 1: K blocks of this launch
  int kb_begin;      // mode 1: first K block of this launch (concatenated over blocks)
  int kb_per_blk;    // mode 1: K blocks per stored block
  int ncols;         // mode 0: B vectors; mode 1: outputs
  int Mvec;          // mode 0: A vectors
  double* part;      // mode 0: [chunk][Mvec][ncols]
  double* Y;         // mode 1
  long long ldy;
  long long L;
  double beta;
  const double* scale;   // mode 1: per output k, alpha 2^(f_k - 42) and alpha 2^(f_k - 63)
  unsigned int* rowmax;   // mode 1, optional: per output k abs_hi of the largest |y|
};

// Tile widths up to 256 columns alternate two TMEM accumulators (a tile's
// epilogue overlaps the next tile's MMAs); the 320-column Gram tile (40
// vectors: the TDHF projections of 20 new vectors in one pass over V) holds
// one 512-column accumulator, issues an N = 256 and an N = 64 MMA per K step
// and loads its B tile as two 160-row boxes.
template <int BN>
struct OzCfg {
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = BN * 128;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE > 8 ? 8 : (200 * 1024) / STAGE;
  static constexpr int NBUF = BN > 256 ? 1 : 2;
  static constexpr int TCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : BN <= 256 ? 256 : 512;
  static constexpr int BOX = BN > 256 ? BN / 2 : BN;   // B rows per TMA box
  static constexpr size_t SMEM = 1024 + static_cast<size_t>(STAGES) * STAGE + (2 * STAGES + 4) * 8 + 16;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Eight float32 accumulators holding exact integers (|v| <= 2^24), weights
// 2^(-7 t) relative to v[0]: split as h = v0 2^28 + v1 2^21 + v2 2^14 + v3 2^7 + v4
// (< 2^53, exact in float64) and g = v5 2^14 + v6 2^7 + v7, formed in integer
// arithmetic; two float64 conversions replace eight float64 multiply-adds.
__device__ __forceinline__ void horner8(const float* v, double& h, double& g) {
  long long hi = __float2int_rn(v[0]);
#pragma unroll
  for (int t = 1; t < 5; ++t) hi = hi * 128 + __float2int_rn(v[t]);
  long long lo = __float2int_rn(v[5]);
  lo = lo * 128 + __float2int_rn(v[6]);
  lo = lo * 128 + __float2int_rn(v[7]);
  h = static_cast<double>(hi);
  g = static_cast<double>(lo);
}

// Persistent kernel: each CTA walks the tiles t = blockIdx.x, + gridDim.x ...;
// the TMA producer streams the K blocks of consecutive tiles through one
// stage ring without draining between tiles, the MMA warp alternates between
// two TMEM accumulators so that the epilogue of one tile overlaps the next.
template <int BN>
__global__ void __launch_bounds__(192, 1)
    oz_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
              const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB, OzArgs a,
              int* err) {
  using C = OzCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ unsigned int kmax[32];   // mode 1 with rowmax: this CTA's per-output maxima
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;    // [2]: accumulator ready for the epilogue
  uint64_t* acce = accf + 2;             // [2]: accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  auto tile_of = [&](int t, int& m0, int& kb0, int& nk, int& kc) {
    if (a.mode == 0) {
      kc = t / a.n_mtiles;
      m0 = (t - kc * a.n_mtiles) * BM;
      kb0 = kc * a.kb_per_cta;
      nk = min(a.kb_per_cta, a.kb_total - kb0);
    } else {
      kc = 0;
      m0 = t * BM;
      kb0 = a.kb_begin;
      nk = a.kb_per_cta;
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, C::NBUF * C::TCOLS);
  if (threadIdx.x < 32) kmax[threadIdx.x] = 0u;
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    long long g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      int m0, kb0, nk, kc;
      tile_of(t, m0, kb0, nk, kc);
      for (int it = 0; it < nk; ++it, ++g) {
        const int s = static_cast<int>(g % C::STAGES);
        if (g >= C::STAGES && !mbar_wait(&empty[s], static_cast<uint32_t>(((g / C::STAGES) + 1) & 1), err, 1)) {
          ok = false;
          break;
        }
        uint8_t* st = base + s * C::STAGE;
        mbar_expect_tx(&full[s], C::STAGE);
        const int kb = kb0 + it;
        if (a.mode == 0) {
          // blocked planes (3-D maps: amplitude in block, plane, block): the
          // tile's planes of one K block are one contiguous read
          tma_load_3d(st, &tmA0, &full[s], 0, m0, kb);
          tma_load_3d(st + C::A_BYTES, &tmB, &full[s], 0, 0, kb);
          if (C::BOX < BN) tma_load_3d(st + C::A_BYTES + C::BOX * 128, &tmB, &full[s], 0, C::BOX, kb);
        } else {
          // blocked nn rows (3-D maps: column in block, amplitude, block): a
          // tile's 128 amplitudes of one column block are one contiguous read
          const int b = kb / a.kb_per_blk;
          const CUtensorMap* ta = b == 0 ? &tmA0 : (b == 1 ? &tmA1 : &tmA2);
          tma_load_3d(st, ta, &full[s], 0, m0, kb - b * a.kb_per_blk);
          tma_load_2d(st + C::A_BYTES, &tmB, &full[s], kb * BKE, 0);
        }
      }
    }
    // the copies still in flight complete before the CTA leaves (bounded)
    for (long long q = (g > C::STAGES ? g - C::STAGES : 0); q < g; ++q)
      mbar_wait(&empty[q % C::STAGES], static_cast<uint32_t>((q / C::STAGES) & 1), err, 0) || true;
  } else if (warp == 1 && lane == 0) {
    // MMA issue (N1 columns, plus N2 more for the 320-column tile)
    constexpr int N1 = BN > 256 ? 256 : BN, N2 = BN - N1;
    constexpr uint32_t idesc = idesc_f32acc(1, BM, N1);
    constexpr uint32_t idesc2 = idesc_f32acc(1, BM, N2 > 0 ? N2 : 16);
    long long g = 0;
    int i = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++i) {
      int m0, kb0, nk, kc;
      tile_of(t, m0, kb0, nk, kc);
      const int buf = i % C::NBUF, use = i / C::NBUF;
      if (use >= 1 && !mbar_wait(&acce[buf], static_cast<uint32_t>((use + 1) & 1), err, 4)) break;
      fence_after_sync();
      const uint32_t acc = tmem + static_cast<uint32_t>(buf * C::TCOLS);
      for (int it = 0; it < nk; ++it, ++g) {
        const int s = static_cast<int>(g % C::STAGES);
        if (!mbar_wait(&full[s], static_cast<uint32_t>((g / C::STAGES) & 1), err, 2)) {
          ok = false;
          break;
        }
        fence_after_sync();
        uint8_t* st = base + s * C::STAGE;
        const uint32_t aa = smem_u32(st), bb = smem_u32(st + C::A_BYTES);
#pragma unroll
        for (int kk = 0; kk < BKE / 16; ++kk) {
          const uint32_t off = kk * 32;   // 16 bf16 per MMA step
          mma_bf16(acc, sdesc(aa + off), sdesc(bb + off), idesc, (it > 0 || kk > 0) ? 1u : 0u);
          if (N2 > 0)
            mma_bf16(acc + N1, sdesc(aa + off), sdesc(bb + N1 * 128 + off), idesc2, (it > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&accf[buf]);
    }
  } else if (warp >= 2) {
    // epilogue: TMEM lanes 32 (warp % 4) .. + 31
    const int q = warp & 3;
    const int r = 32 * q + lane;
    int i = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++i) {
      int m0, kb0, nk, kc;
      tile_of(t, m0, kb0, nk, kc);
      const int buf = i % C::NBUF;
      if (!mbar_wait(&accf[buf], static_cast<uint32_t>((i / C::NBUF) & 1), err, 3)) break;
      fence_after_sync();
      const uint32_t trow = tmem + static_cast<uint32_t>(buf * C::TCOLS) + (static_cast<uint32_t>(32 * q) << 16);
      if (a.mode == 0) {
        // row r = digit plane i of vector m0/8 + r/8; column n*8 + j
        const int di = r & 7;
        const double c1 = ldexp(1.0, -35 - 7 * (di + 1)), c2 = ldexp(1.0, -56 - 7 * (di + 1));
        const int mv = (m0 + r) >> 3;
        double* out = a.part + (static_cast<size_t>(kc) * a.Mvec + mv) * a.ncols;
        for (int n = 0; n < a.ncols; ++n) {
          float v[8];
          tmem_ld8(trow + n * 8, v);
          double h, gg;
          horner8(v, h, gg);
          double sum = fma(h, c1, gg * c2);
          sum += __shfl_xor_sync(0xffffffffu, sum, 1);
          sum += __shfl_xor_sync(0xffffffffu, sum, 2);
          sum += __shfl_xor_sync(0xffffffffu, sum, 4);
          if ((lane & 7) == 0 && mv < a.Mvec) out[n] = sum;
        }
      } else {
        const long long l = static_cast<long long>(m0) + r;
        for (int k = 0; k < a.ncols; ++k) {
          float v[8];
          tmem_ld8(trow + k * 8, v);
          unsigned int ym = 0;
          if (l < a.L) {
            double h, gg;
            horner8(v, h, gg);
            double y = fma(h, a.scale[2 * k], gg * a.scale[2 * k + 1]);
            double* p = a.Y + static_cast<size_t>(k) * a.ldy + l;
            if (a.beta != 0.0) y = fma(a.beta, *p, y);
            *p = y;
            ym = abs_hi(y);
          }
          if (a.rowmax) {   // the output's largest |y|: per CTA in shared memory, flushed at exit
            ym = __reduce_max_sync(0xffffffffu, ym);
            if (lane == 0 && ym) atomicMax(&kmax[k], ym);
          }
        }
      }
      fence_before_sync();
      mbar_arrive(&acce[buf]);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, C::NBUF * C::TCOLS);
  }
  if (a.mode == 1 && a.rowmax && threadIdx.x < a.ncols && kmax[threadIdx.x])
    atomicMax(&a.rowmax[threadIdx.x], kmax[threadIdx.x]);
}

// abs_hi of the largest |x| of each row (common.cuh: the high word of the
// bit pattern, ordered like |x|); four independent loads in flight per thread
__global__ void oz_absmax_kernel(long long L, const double* __restrict__ X, long long ldx,
                                 unsigned int* __restrict__ mx) {
  const int r = blockIdx.y;
  const double* x = X + static_cast<size_t>(r) * ldx;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  unsigned int m0 = 0, m1 = 0, m2 = 0, m3 = 0;
  long long l = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; l + 3 * stride < L; l += 4 * stride) {
    const double a = x[l], b = x[l + stride], c = x[l + 2 * stride], d = x[l + 3 * stride];
    m0 = max(m0, abs_hi(a));
    m1 = max(m1, abs_hi(b));
    m2 = max(m2, abs_hi(c));
    m3 = max(m3, abs_hi(d));
  }
  for (; l < L; l += stride) m0 = max(m0, abs_hi(x[l]));
  unsigned int m = __reduce_max_sync(0xffffffffu, max(max(m0, m1), max(m2, m3)));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&mx[r], m);
}

// exponents from abs_hi row maxima: max |x| < 2^(e-1), e = 0 for an all-zero
// (or subnormal) row; a non-finite maximum raises the error word (code 10)
__global__ void oz_exp_kernel(int nvec, const unsigned int* __restrict__ mx, int* __restrict__ e, int* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nvec) return;
  const unsigned int hw = mx[r];
  const int ex = static_cast<int>((hw >> 20) & 0x7FF);
  if (ex == 0x7FF) atomicCAS(err, 0, 10);
  e[r] = (ex == 0) ? 0 : ex - 1021;
}

// One CTA per 64 consecutive amplitudes l and up to 32 vectors: digits are
// formed with l along the threads (coalesced float64 loads and tn plane
// stores) and staged in shared memory, then the nn rows are written with the
// vectors along the threads, so each row's nvec x 16 bytes go out contiguously.
constexpr int kSliceL = 64, kSliceR = 32;

__global__ void __launch_bounds__(256) oz_slice_kernel(int nvec, long long L, const double* __restrict__ X,
                                                       long long ldx, const int* __restrict__ e,
                                                       oz_t* __restrict__ tn, long long Lp, long long P,
                                                       int tn_r0, oz_t* __restrict__ nn, int ldk, int nn_r0) {
  __shared__ uint4 tile[kSliceR][kSliceL];
  const long long l0 = static_cast<long long>(blockIdx.x) * kSliceL;
  const int r0 = blockIdx.y * kSliceR;
  const int nr = min(kSliceR, nvec - r0);
  // each thread splits two consecutive amplitudes, so every tn plane gets one
  // 4-byte store per pair (the pair's first index is even and shares its
  // 64-amplitude block)
  constexpr int kPairs = kSliceL / 2;
  for (int item = threadIdx.x; item < nr * kPairs; item += blockDim.x) {
    const int r = item / kPairs, li = 2 * (item % kPairs);
    const long long l = l0 + li;
    const int rv = r0 + r;
    int d0[kOzDigits], d1[kOzDigits];
    const double* xr = X + static_cast<size_t>(rv) * ldx;
    if (l < L) {
      oz_digits(xr[l], e[rv], d0);
    } else {
#pragma unroll
      for (int i = 0; i < kOzDigits; ++i) d0[i] = 0;
    }
    if (l + 1 < L) {
      oz_digits(xr[l + 1], e[rv], d1);
    } else {
#pragma unroll
      for (int i = 0; i < kOzDigits; ++i) d1[i] = 0;
    }
    if (tn && l < Lp) {
#pragma unroll
      for (int i = 0; i < kOzDigits; ++i) {
        const uint32_t two = static_cast<uint32_t>(digit_bits(d0[i])) | (static_cast<uint32_t>(digit_bits(d1[i])) << 16);
        const size_t p = static_cast<size_t>(tn_r0 + rv) * kOzDigits + i;
        *reinterpret_cast<uint32_t*>(tn + ((static_cast<size_t>(l >> 6) * P + p) << 6) + (l & 63)) = two;
      }
    }
    if (nn) {
      tile[r][li] = pack8(d0);
      tile[r][li + 1] = pack8(d1);
    }
  }
  if (!nn) return;
  __syncthreads();
  for (int item = threadIdx.x; item < kSliceL * nr; item += blockDim.x) {
    const int li = item / nr, r = item % nr;
    const long long l = l0 + li;
    if (l < L) {
      const size_t k = static_cast<size_t>(nn_r0 + r0 + r) * kOzDigits;   // 64-column blocks, all amplitudes each
      *reinterpret_cast<uint4*>(nn + (((k >> 6) * L + l) << 6) + (k & 63)) = tile[r][li];
    }
  }
}

// C[m][n] = alpha 2^(eA[m] + eB[n]) sum_chunk part[chunk][m][n] + beta C[m][n];
// one warp per output: lane-strided partial sums, then a fixed shuffle tree
// (the same order on every run)
__global__ void oz_reduce_kernel(int M, int N, int nchunk, const double* __restrict__ part, const int* __restrict__ eA,
                                 const int* __restrict__ eB, double alpha, double beta, double* C, int ldc) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= M * N) return;
  const int m = w / N, n = w % N;
  double sum = 0.0;
  for (int c = lane; c < nchunk; c += 32) sum += part[(static_cast<size_t>(c) * M + m) * N + n];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    double y = alpha * ldexp(sum, eA[m] + eB[n]);
    double* p = C + static_cast<size_t>(m) * ldc + n;
    if (beta != 0.0) y = fma(beta, *p, y);
    *p = y;
  }
}

struct CoefArgs {
  const double* coef[3];
  int ldc[3];
  const int* e[3];
};

// Digit matrix of the combination coefficients, one CTA per output k:
// column (k, t) of the product (row k * 8 + t here, K-major over the
// concatenated blocks) holds at K index (b, m, i) the digit t - i of
// c'[b][m] = coef_b[m][k] 2^(e_b[m]), split with the common exponent f[k].
__global__ void oz_coef_kernel(int nb, int S, int Kp, int k0, CoefArgs ca, double alpha, oz_t* __restrict__ bmat,
                               double* __restrict__ scale, int* err) {
  const int k = blockIdx.x;
  const int rowK = nb * Kp;
  const int per = Kp / kOzDigits;
  __shared__ unsigned long long smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  unsigned long long mx = 0;
  for (int idx = threadIdx.x; idx < nb * S; idx += blockDim.x) {
    const int b = idx / S, m = idx % S;
    const double c = ldexp(ca.coef[b][static_cast<size_t>(m) * ca.ldc[b] + k0 + k], ca.e[b][m]);
    mx = max(mx, static_cast<unsigned long long>(__double_as_longlong(fabs(c))));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, mx);
  __syncthreads();
  const unsigned long long M = smax;
  const int ex = static_cast<int>((M >> 52) & 0x7FF);
  if (threadIdx.x == 0 && ex == 0x7FF) atomicCAS(err, 0, 11);
  const int f = (M == 0) ? 0 : ex - 1021;
  if (threadIdx.x == 0) {
    // output weights of the anti-diagonal sums split as in horner8
    scale[2 * k] = alpha * ldexp(1.0, f - 42);
    scale[2 * k + 1] = alpha * ldexp(1.0, f - 63);
  }
  for (int idx = threadIdx.x; idx < nb * per; idx += blockDim.x) {
    const int b = idx / per, m = idx % per;
    int d[kOzDigits];
    if (m < S) {
      oz_digits(ldexp(ca.coef[b][static_cast<size_t>(m) * ca.ldc[b] + k0 + k], ca.e[b][m]), f, d);
    } else {
#pragma unroll
      for (int i = 0; i < kOzDigits; ++i) d[i] = 0;
    }
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) {
      int g[kOzDigits];
#pragma unroll
      for (int i = 0; i < kOzDigits; ++i) g[i] = (i <= t) ? d[t - i] : 0;
      *reinterpret_cast<uint4*>(bmat + static_cast<size_t>(k * kOzDigits + t) * rowK + static_cast<size_t>(b) * Kp +
                                static_cast<size_t>(m) * kOzDigits) = pack8(g);
    }
  }
}

// inner x rows bf16 matrix, row stride ld elements, boxes of 64 x box_rows
// tn digit planes (oz_slice): rows planes of a blocked array with plane
// capacity P, nblk blocks of 64 amplitudes; box = 64 amplitudes x box_rows
// planes of one block
CUtensorMap make_map_planes(const oz_t* ptr, long long rows, long long P, long long nblk, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(BKE), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(nblk)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(BKE) * 2, static_cast<cuuint64_t>(P) * BKE * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(BKE), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || rows <= 0 || nblk <= 0 || P < rows)
    throw Error(XS_EINVAL, "digit planes not 16-byte aligned, empty or beyond their capacity");
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<oz_t*>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(XS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
  return m;
}

CUtensorMap make_map_bf16(const oz_t* ptr, long long inner, long long rows, long long ld, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(BKE), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld % 8) || inner <= 0 || rows <= 0)
    throw Error(XS_EINVAL, "digit operand not 16-byte aligned or empty");
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<oz_t*>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(XS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
  return m;
}

int num_sms() {
  static const int n = [] {
    int dev = 0, count = 0;
    XS_CUDA(cudaGetDevice(&dev));
    XS_CUDA(cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev));
    return count;
  }();
  return n;
}

template <int BN>
void launch_oz(cudaStream_t s, const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& a2,
               const CUtensorMap& b, const OzArgs& args, int* err) {
  using C = OzCfg<BN>;
  static const bool attr = [] {   // once per process (thread-safe initialisation)
    XS_CUDA(cudaFuncSetAttribute(oz_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(C::SMEM)));
    return true;
  }();
  (void)attr;
  const int grid = std::min(args.ntiles, num_sms());   // persistent: one CTA per SM
  oz_kernel<BN><<<grid, 192, C::SMEM, s>>>(a0, a1, a2, b, args, err);
  XS_CHECK_LAUNCH();
}

int pick_bn(int cols) { return cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 192 ? 192 : cols <= 256 ? 256 : 320; }

void dispatch(cudaStream_t s, int bn, const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& a2,
              const CUtensorMap& b, const OzArgs& args, int* err) {
  switch (bn) {
    case 64: launch_oz<64>(s, a0, a1, a2, b, args, err); break;
    case 128: launch_oz<128>(s, a0, a1, a2, b, args, err); break;
    case 192: launch_oz<192>(s, a0, a1, a2, b, args, err); break;
    case 256: launch_oz<256>(s, a0, a1, a2, b, args, err); break;
    default: launch_oz<320>(s, a0, a1, a2, b, args, err); break;
  }
}

constexpr int kMaxCols = 256 / kOzDigits;       // outputs of a combination per launch
constexpr int kMaxGramCols = 320 / kOzDigits;   // B vectors of a Gram per launch

}  // namespace

void oz_exponents_from_max(cudaStream_t s, int nvec, const unsigned int* mx, int* e, int* err) {
  if (nvec <= 0) return;
  oz_exp_kernel<<<(nvec + 127) / 128, 128, 0, s>>>(nvec, mx, e, err);
  XS_CHECK_LAUNCH();
}

void oz_exponents(cudaStream_t s, int nvec, long long L, const double* X, long long ldx, int* e, OzWork& w,
                  int* err) {
  if (nvec <= 0) return;
  ProfScope ps(s, "oz_exponents", 8.0 * nvec * L, 0.0);
  w.mx.ensure(nvec);
  XS_CUDA(cudaMemsetAsync(w.mx.get(), 0, sizeof(unsigned int) * nvec, s));
  if (L > 0) {
    // about 8 CTAs per SM over all rows, at least 1024 amplitudes per CTA
    const long long per_row = std::max<long long>(1, std::min<long long>((8LL * 152 + nvec - 1) / nvec, (L + 1023) / 1024));
    dim3 grid(static_cast<unsigned>(per_row), nvec);
    oz_absmax_kernel<<<grid, 256, 0, s>>>(L, X, ldx, w.mx.get());
    XS_CHECK_LAUNCH();
  }
  oz_exp_kernel<<<(nvec + 127) / 128, 128, 0, s>>>(nvec, w.mx.get(), e, err);
  XS_CHECK_LAUNCH();
}

void oz_slice(cudaStream_t s, int nvec, long long L, const double* X, long long ldx, const int* e, oz_t* tn,
              long long P, int tn_r0, oz_t* nn, int ldk, int nn_r0) {
  if (nvec <= 0 || (!tn && !nn)) return;
  const long long Lp = oz_lp(L);
  if (tn && P < static_cast<long long>(tn_r0 + nvec) * kOzDigits) throw Error(XS_EINVAL, "oz_slice: plane capacity");
  if (nn && (ldk % 64 || static_cast<long long>(nn_r0 + nvec) * kOzDigits > ldk))
    throw Error(XS_EINVAL, "oz_slice: nn column capacity");
  const long long span = tn ? Lp : L;
  ProfScope ps(s, "oz_slice", 8.0 * nvec * L + (tn ? 16.0 * nvec * Lp : 0.0) + (nn ? 16.0 * nvec * L : 0.0), 0.0);
  dim3 grid(static_cast<unsigned>((span + kSliceL - 1) / kSliceL), (nvec + kSliceR - 1) / kSliceR);
  oz_slice_kernel<<<grid, 256, 0, s>>>(nvec, L, X, ldx, e, tn, Lp, P, tn_r0, nn, ldk, nn_r0);
  XS_CHECK_LAUNCH();
}

void oz_gram(cudaStream_t s, int M, int N, long long L, const oz_t* Atn, long long AP, const int* eA,
             const oz_t* Btn, long long BP, const int* eB, double alpha, double beta, double* C, int ldc,
             OzWork& w, int* err) {
  if (M <= 0 || N <= 0) return;
  if (L <= 0) throw Error(XS_EINVAL, "oz_gram: empty vectors");
  const int kb_total = static_cast<int>((L + BKE - 1) / BKE);
  const int nchunk = (kb_total + KB_CHUNK - 1) / KB_CHUNK;
  const long long nblk = oz_lp(L) / BKE;
  const CUtensorMap ta = make_map_planes(Atn, static_cast<long long>(M) * kOzDigits, AP, nblk, BM);
  for (int n0 = 0; n0 < N; n0 += kMaxGramCols) {
    const int nn = std::min(kMaxGramCols, N - n0);
    const int bn = pick_bn(nn * kOzDigits);
    // B planes n0 * 8.. of every block: the map starts n0 * 8 planes into block 0
    const CUtensorMap tb = make_map_planes(Btn + static_cast<size_t>(n0) * kOzDigits * BKE,
                                           static_cast<long long>(nn) * kOzDigits, BP, nblk, bn > 256 ? bn / 2 : bn);
    w.part.ensure(static_cast<size_t>(nchunk) * M * nn);
    OzArgs a{};
    a.mode = 0;
    a.n_mtiles = (M * kOzDigits + BM - 1) / BM;
    a.ntiles = a.n_mtiles * nchunk;
    a.kb_total = kb_total;
    a.kb_per_cta = KB_CHUNK;
    a.ncols = nn;
    a.Mvec = M;
    a.part = w.part.get();
    {
      ProfScope ps(s, "oz_gram", 2.0 * kOzDigits * static_cast<double>(L) * (M + nn), 2.0 * M * nn * (double)L);
      dispatch(s, bn, ta, ta, ta, tb, a, err);
    }
    oz_reduce_kernel<<<grid1(32LL * M * nn, 256), 256, 0, s>>>(M, nn, nchunk, w.part.get(), eA, eB + n0, alpha, beta,
                                                                C + n0, ldc);
    XS_CHECK_LAUNCH();
  }
}

void oz_combine(cudaStream_t s, int nb, const OzBlock* blk, int S, int nout, long long L, double alpha, double beta,
                double* Y, long long ldy, OzWork& w, int* err, unsigned int* rowmax) {
  if (nout <= 0 || L <= 0) return;
  if (rowmax) XS_CUDA(cudaMemsetAsync(rowmax, 0, sizeof(unsigned int) * nout, s));
  if (nb < 1 || nb > 3) throw Error(XS_EINVAL, "oz_combine: 1 to 3 blocks");
  if (S <= 0) throw Error(XS_EINVAL, "oz_combine: empty subspace");
  const int Kp = oz_ldk(S);
  const int kb_per_blk = Kp / BKE;
  const int kb_total = nb * kb_per_blk;
  CUtensorMap ta[3];
  CoefArgs ca{};
  for (int b = 0; b < nb; ++b) {
    if (blk[b].ldk < Kp || blk[b].ldk % 64) throw Error(XS_EINVAL, "oz_combine: nn capacity too small");
    // the first Kp / 64 column blocks of L amplitudes each (the same 3-D form as the tn planes)
    ta[b] = make_map_planes(blk[b].nn, L, L, Kp / BKE, BM);
    ca.coef[b] = blk[b].coef;
    ca.ldc[b] = blk[b].ldc;
    ca.e[b] = blk[b].e;
  }
  for (int b = nb; b < 3; ++b) ta[b] = ta[0];
  for (int k0 = 0; k0 < nout; k0 += kMaxCols) {
    const int nk = std::min(kMaxCols, nout - k0);
    const int bn = pick_bn(nk * kOzDigits);
    w.bmat.ensure(static_cast<size_t>(nk) * kOzDigits * nb * Kp);
    w.scale.ensure(2 * kMaxCols);
    oz_coef_kernel<<<nk, 256, 0, s>>>(nb, S, Kp, k0, ca, alpha, w.bmat.get(), w.scale.get(), err);
    XS_CHECK_LAUNCH();
    const CUtensorMap tb = make_map_bf16(w.bmat.get(), static_cast<long long>(nb) * Kp,
                                         static_cast<long long>(nk) * kOzDigits, static_cast<long long>(nb) * Kp, bn);
    for (int kb = 0; kb < kb_total; kb += KB_CHUNK) {
      OzArgs a{};
      a.mode = 1;
      a.ntiles = static_cast<int>((L + BM - 1) / BM);
      a.kb_begin = kb;
      a.kb_per_cta = std::min(KB_CHUNK, kb_total - kb);
      a.kb_per_blk = kb_per_blk;
      a.ncols = nk;
      a.Y = Y + static_cast<size_t>(k0) * ldy;
      a.ldy = ldy;
      a.L = L;
      a.beta = kb == 0 ? beta : 1.0;
      a.scale = w.scale.get();
      a.rowmax = (rowmax && kb + KB_CHUNK >= kb_total) ? rowmax + k0 : nullptr;
      ProfScope ps(s, "oz_combine",
                   2.0 * kOzDigits * static_cast<double>(L) * a.kb_per_cta * BKE / kOzDigits +
                       8.0 * nk * (double)L * (a.beta != 0.0 ? 2 : 1),
                   2.0 * nk * (double)L * a.kb_per_cta * BKE / kOzDigits);
      dispatch(s, bn, ta[0], ta[1], ta[2], tb, a, err);
    }
  }
}

}  // namespace xs
