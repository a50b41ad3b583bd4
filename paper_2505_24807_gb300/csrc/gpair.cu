// Float32 G(R) build over unordered pairs of super-atoms (the G build of the
// mixed-precision products; paper, Section "GPU Implementation", Eq. ftilde).
//
// A super-atom is a heavy atom (4 AOs) or a run of up to 4 consecutive
// hydrogens.  One thread owns one unordered pair (I, J) of super-atoms: it
// loads the pair's two-centre integrals (mu nu|lam sig) once into shared
// memory (at most 10 x 10 products) and then, for every matrix of the batch, reads
// the two 4 x 4 blocks R_IJ and R_JI once, forms both exchange blocks
//   K_IJ[mu][lam] = sum_{nu in at(mu), sig in at(lam)} (mu nu|lam sig) R[nu][sig]
//   K_JI[lam][mu] = sum (mu nu|lam sig) R[sig][nu]
// and writes both G blocks.  Because K(R^T)_IJ = K_JI^T, the TDHF outputs
// need no second pass over R:
//   CIS:  G_IJ = -K_IJ,                G_JI = -K_JI
//   TDHF: G+_IJ = -(K_IJ + K_JI^T),    G+_JI = G+_IJ^T
//         G-_IJ = -(K_IJ - K_JI^T),    G-_JI = -G-_IJ^T
// Pairs with I = J hold the diagonal atom blocks: the closed-form one-centre
// Coulomb and exchange terms, the two-centre Coulomb J2 = W r of the diagonal
// blocks, and inside a hydrogen run the exchange between its hydrogens.
// Every R element is read once and every G element written once per matrix.
// A warp holds 2 consecutive super-atoms I x 16 consecutive super-atoms J, so
// the row segments it reads and writes are contiguous (16-byte loads and
// stores where the blocks start on multiples of 4 AOs), and each thread keeps
// the next matrix's blocks in flight while it contracts the current one.
#include <vector>

#include "gpair_dev.cuh"
#include "kernels.h"
#include "prof.h"

namespace xs {

namespace {

constexpr int kPairThreads = 256;

template <GMode MODE, bool SPLIT>
__global__ void __launch_bounds__(kPairThreads, 2) gpair_kernel(int n, int np, int nvec, int npairs,
                                                                const int2* __restrict__ pairs,
                                                                const int4* __restrict__ sa,
                                                                const double* __restrict__ par,
                                                                const float* __restrict__ W,
                                                                const float* __restrict__ J2, int ldj,
                                                                const float* __restrict__ R, PairOut o) {
  extern __shared__ float wsm[];   // 100 integrals per thread
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npairs) return;
  gpair_one<MODE, SPLIT>(n, np, nvec, pairs[t], sa, par, W, J2, ldj, R, o, wsm + threadIdx.x * 100);
}

template <bool SPLIT>
void launch_pairs(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* W,
                  const float* J2, int ldj, const float* R, const PairOut& o) {
  const int np2 = m.gp_npairs;
  const int2* pairs = reinterpret_cast<const int2*>(m.gp_pairs.get());
  const int4* sa = reinterpret_cast<const int4*>(m.gp_sa.get());
  const dim3 grid((np2 + kPairThreads - 1) / kPairThreads);
  const size_t smem = sizeof(float) * 100 * kPairThreads;
  static const bool attr = [] {
    for (const void* f : {reinterpret_cast<const void*>(gpair_kernel<G_CIS, SPLIT>),
                          reinterpret_cast<const void*>(gpair_kernel<G_RPA, SPLIT>),
                          reinterpret_cast<const void*>(gpair_kernel<G_CIS_T, SPLIT>),
                          reinterpret_cast<const void*>(gpair_kernel<G_RPA_T, SPLIT>)})
      XS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(float) * 100 * kPairThreads)));
    return true;
  }();
  (void)attr;
  switch (mode) {
    case G_CIS:
      gpair_kernel<G_CIS, SPLIT><<<grid, kPairThreads, smem, s>>>(m.n, m.np, nvec, np2, pairs, sa, d_par, W, J2, ldj, R, o);
      break;
    case G_RPA:
      gpair_kernel<G_RPA, SPLIT><<<grid, kPairThreads, smem, s>>>(m.n, m.np, nvec, np2, pairs, sa, d_par, W, J2, ldj, R, o);
      break;
    case G_CIS_T:
      gpair_kernel<G_CIS_T, SPLIT><<<grid, kPairThreads, smem, s>>>(m.n, m.np, nvec, np2, pairs, sa, d_par, W, J2, ldj, R, o);
      break;
    default:
      gpair_kernel<G_RPA_T, SPLIT><<<grid, kPairThreads, smem, s>>>(m.n, m.np, nvec, np2, pairs, sa, d_par, W, J2, ldj, R, o);
      break;
  }
  XS_CHECK_LAUNCH();
}

// Two-centre Coulomb of the diagonal blocks, J2 = W r (np x nvec, row
// stride nvec), W symmetric np x np, r np x nvec (row stride nvec).
// W is streamed once: J2[q][v] = sum_p W[p][q] r[p][v], threads along q (row
// segments of W), CTAs along q blocks and p chunks; the chunk partials are
// summed in chunk order (deterministic).
constexpr int kJ2Rows = 128;   // p rows per chunk
constexpr int kJ2Vec = 16;     // vectors per pass

__global__ void __launch_bounds__(256) j2_partial_kernel(int np, int nvec, const float* __restrict__ W,
                                                         const float* __restrict__ r, float* __restrict__ part) {
  __shared__ float rs[kJ2Rows][kJ2Vec];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p0 = blockIdx.y * kJ2Rows, p1 = min(np, p0 + kJ2Rows);
  for (int v0 = 0; v0 < nvec; v0 += kJ2Vec) {
    const int nv = min(kJ2Vec, nvec - v0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kJ2Rows * kJ2Vec; idx += blockDim.x) {
      const int pp = idx / kJ2Vec, v = idx - pp * kJ2Vec;
      rs[pp][v] = (p0 + pp < p1 && v < nv) ? r[(long long)(p0 + pp) * nvec + v0 + v] : 0.0f;
    }
    __syncthreads();
    if (q < np) {
      float acc[kJ2Vec];
#pragma unroll
      for (int v = 0; v < kJ2Vec; ++v) acc[v] = 0.0f;
      for (int p = p0; p < p1; ++p) {
        const float w = __ldg(W + (long long)p * np + q);
#pragma unroll
        for (int v = 0; v < kJ2Vec; ++v) acc[v] = fmaf(w, rs[p - p0][v], acc[v]);
      }
      float* out = part + ((long long)blockIdx.y * np + q) * nvec + v0;
      for (int v = 0; v < nv; ++v) out[v] = acc[v];
    }
  }
}

__global__ void j2_reduce_kernel(int np, int nvec, int nchunk, const float* __restrict__ part, float* __restrict__ J2) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)np * nvec) return;
  float s = 0.0f;
  for (int c = 0; c < nchunk; ++c) s += part[(long long)c * np * nvec + idx];
  J2[idx] = s;
}

}  // namespace

void build_gpairs(cudaStream_t s, DevMol& m) {
  const MolLayout& L = m.L;
  std::vector<int> sa;   // x, y, z, w per super-atom
  for (int A = 0; A < L.natoms;) {
    if (L.nao_atom[A] == 4) {
      sa.insert(sa.end(), {L.ao_off[A], 4 | 16, L.prod_off[A], L.elem[A]});
      ++A;
      continue;
    }
    int A1 = A, cnt = 0;
    while (A1 < L.natoms && L.nao_atom[A1] == 1 && cnt < 4) { ++A1; ++cnt; }
    sa.insert(sa.end(), {L.ao_off[A], cnt, L.prod_off[A], L.elem[A]});
    A = A1;
  }
  const int ns = static_cast<int>(sa.size() / 4);
  // warp blocks: 2 consecutive super-atoms I x 16 consecutive super-atoms J >= I
  std::vector<int> pairs;
  for (int I0 = 0; I0 < ns; I0 += 2)
    for (int J0 = (I0 / 16) * 16; J0 < ns; J0 += 16) {
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 16; ++b) {
          const int I = I0 + a, J = J0 + b;
          const bool ok = I < ns && J < ns && J >= I;
          pairs.push_back(ok ? I : -1);
          pairs.push_back(ok ? J : -1);
        }
    }
  m.gp_nsa = ns;
  m.gp_npairs = static_cast<int>(pairs.size() / 2);
  m.gp_sa.alloc(sa.size());
  m.gp_pairs.alloc(pairs.size());
  XS_CUDA(cudaMemcpyAsync(m.gp_sa.get(), sa.data(), sizeof(int) * sa.size(), cudaMemcpyHostToDevice, s));
  XS_CUDA(cudaMemcpyAsync(m.gp_pairs.get(), pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, s));
  XS_CUDA(cudaStreamSynchronize(s));
}

void coulomb_j2(cudaStream_t s, int np, int nvec, const float* W, const float* r, float* J2, DevBuf<float>& ws) {
  if (nvec <= 0) return;
  const int nchunk = (np + kJ2Rows - 1) / kJ2Rows;
  ws.ensure((size_t)nchunk * np * nvec);
  ProfScope ps(s, "coulomb_j2_f32", 4.0 * ((double)np * np + 2.0 * np * nvec), 2.0 * (double)np * np * nvec);
  j2_partial_kernel<<<dim3((np + 255) / 256, nchunk), 256, 0, s>>>(np, nvec, W, r, ws.get());
  XS_CHECK_LAUNCH();
  j2_reduce_kernel<<<grid1((long long)np * nvec, 256), 256, 0, s>>>(np, nvec, nchunk, ws.get(), J2);
  XS_CHECK_LAUNCH();
}

void gpair_build(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* W,
                 const float* J2, int ldj, const float* R, float* G, float* Gm) {
  PairOut o{G, Gm, nullptr, nullptr, nullptr, nullptr, 0};
  launch_pairs<false>(s, m, d_par, mode, nvec, W, J2, ldj, R, o);
}

void gpair_build_split(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* W,
                       const float* J2, int ldj, const float* R, float* Gh, float* Gl, float* Gmh, float* Gml,
                       int ldo) {
  PairOut o{nullptr, nullptr, Gh, Gl, Gmh, Gml, ldo};
  launch_pairs<true>(s, m, d_par, mode, nvec, W, J2, ldj, R, o);
}

}  // namespace xs
