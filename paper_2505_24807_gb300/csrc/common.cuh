// Shared definitions of libxs's CUDA sources: status plumbing, device
// buffers, per-molecule device state and the context.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/xs.h"
#include "model.h"
#include "prof.h"

namespace xs {

#ifdef __CUDACC__
// High 32 bits of |x|'s bit pattern (sign cleared: exponent and the top 20
// mantissa bits).  Ordered like |x| and enough for its binary exponent: the
// per-row maxima that set the digit exponents of the Davidson subspace.
__device__ __forceinline__ unsigned int abs_hi(double x) {
  return static_cast<unsigned int>(static_cast<unsigned long long>(__double_as_longlong(x)) >> 32) & 0x7FFFFFFFu;
}
#endif
struct Mlp;
}

namespace xs {

// Errors inside the library are C++ exceptions carrying a status; the C ABI
// layer catches them, stores the message and returns the status.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define XS_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw ::xs::Error(e_ == cudaErrorMemoryAllocation ? XS_ENOMEM : XS_ECUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

#define XS_CHECK_LAUNCH()                                   \
  do {                                                      \
    XS_CUDA(cudaGetLastError());                            \
    if (::xs::g_prof && ::xs::g_prof->on) ++::xs::g_prof->launches; \
  } while (0)

// Owning device buffer.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    if (count == n && p) return;
    release();
    if (count) XS_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void ensure(size_t count) { if (count > n) alloc(count); }
  void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
  T* get() const { return p; }
};

// Device copy of one molecule's ground state and integrals.
struct DevMol {
  MolLayout L;
  int n = 0, o = 0, v = 0, np = 0;
  DevBuf<int> ao_atom, ao_local, atom_ao_off, atom_nao, atom_prod_off, atom_elem;
  DevBuf<double> xyz;     // atoms x 3
  DevBuf<double> W;       // np x np two-centre supermatrix (float64)
  DevBuf<float> Wf;       // float32 copy for the mixed path
  DevBuf<double> H;       // core Hamiltonian n x n
  DevBuf<double> CT;      // MO coefficients, MO-major: CT[p * n + mu] = C[mu][p]
  DevBuf<double> eps;     // n orbital energies
  DevBuf<float> CTf_hi, CTf_lo;  // TF32-pair operand copies of CT for the tensor-core path
  DevBuf<float> CTf;             // float32 copy of CT for the float32 SIMT products
  DevBuf<double> dip;            // MO dipole integrals <i|r_x|a>, 3 x nocc x nvir (lazily)
  DevBuf<int> gb_rows, gb_cols;  // atom-aligned G tiles (first AO, count, first atom, end atom)
  int gb_nrows = 0, gb_ncols = 0;
  DevBuf<int> gp_sa, gp_pairs;   // super-atoms (int4) and unordered super-atom pairs (int2) of the float32 G build
  int gp_nsa = 0, gp_npairs = 0;
  bool ready = false;
  int scf_iterations = 0;
  // last excited-state solution
  int nroots = 0, method = 0, spin = 0;
  DevBuf<double> U, Wv;   // nroots x ov: X+Y and X-Y (CIS: X and X)
  std::vector<double> omega, osc, resid;
  int iterations = 0;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  ElemParams par[XS_NELEM];
  bool have_params = false;
  std::vector<DevMol> mols;
  DevBuf<double> d_par;   // XS_NELEM x XS_NPARAM on the device
  void* solver = nullptr; // cusolverDnHandle_t, created on first use
  // scratch reused across calls
  DevBuf<double> ws0, ws1, ws2, ws3, ws4, ws5;
  DevBuf<float> fs0, fs1, fs2;
  Profiler prof;
  DevBuf<int> tc_err;   // error word of the tensor-core kernels' bounded waits
  std::shared_ptr<void> dav_cache;  // Davidson workspace kept between solves (davidson.cu)
  std::shared_ptr<void> batch_cache;  // lock-step batched solver's arenas (batch.cu)
  // batched solves: worker contexts (own stream and scratch), reused across calls
  std::vector<std::unique_ptr<Ctx>> workers;
  // learned guess / preconditioner network (shared by the workers)
  std::shared_ptr<Mlp> mlp;
};

inline dim3 grid1(long long n, int block) { return dim3(static_cast<unsigned>((n + block - 1) / block)); }

}  // namespace xs

struct xs_ctx {
  xs::Ctx c;
};
