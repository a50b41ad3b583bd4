// Allocation-free G(R) build (declared in include/xs.h as xs_gbuild_noalloc).
//
// For callers that cannot call cudaMalloc while they call into the library --
// a process whose device memory is reserved up front by another allocator's
// pool, or a latency-critical loop that must not meet cudaMalloc's implicit
// device synchronisation -- the two scratch vectors of the G build (packed
// diagonal blocks r and the Coulomb products J2) come from one fixed array
// compiled into the library instead of from cudaMalloc.  The kernels are the
// ones the allocating path launches.
#include <mutex>
#include <vector>

#include "kernels.h"

namespace {

// np * nvec doubles for r plus as many for J2; 2^18 doubles = 2 MiB, held by
// every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 18;
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mutex;
std::vector<double*> g_noalloc_ptr;  // per device: device address of g_noalloc_scratch

// Device address of the scratch array on `device` (the current device), looked
// up once per device; the host-side symbol itself is not a device address.
double* noalloc_scratch(int device) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (device >= static_cast<int>(g_noalloc_ptr.size())) g_noalloc_ptr.resize(device + 1, nullptr);
  if (!g_noalloc_ptr[device]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
    if (e != cudaSuccess)
      throw xs::Error(XS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  return g_noalloc_ptr[device];
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int xs_gbuild_noalloc(xs_ctx* ctx, int mol, int nvec, const double* R, double* G) {
  if (!ctx) return XS_EINVAL;
  xs::Ctx& c = ctx->c;
  c.err.clear();
  try {
    XS_CUDA(cudaSetDevice(c.device));
    if (mol < 0 || mol >= static_cast<int>(c.mols.size()) || !c.mols[mol].ready)
      throw xs::Error(XS_ESTATE, "molecule has no ground state");
    const xs::DevMol& m = c.mols[mol];
    if (nvec < 0) throw xs::Error(XS_EINVAL, "nvec must be >= 0");
    if (nvec == 0) return XS_OK;
    const size_t need = 2 * static_cast<size_t>(m.np) * static_cast<size_t>(nvec);
    if (need > kNoAllocScratchDoubles)
      throw xs::Error(XS_EINVAL, "xs_gbuild_noalloc: 2 * nprod * nvec = " + std::to_string(need) +
                                     " doubles exceeds the fixed scratch of " +
                                     std::to_string(kNoAllocScratchDoubles) + "; use fewer vectors per call");
    if (!R || !G || !is_device_pointer(R) || !is_device_pointer(G))
      throw xs::Error(XS_EINVAL, "xs_gbuild_noalloc: R and G must be device pointers");
    double* scratch = noalloc_scratch(c.device);
    xs::NoTuneScope no_tune;
    xs::gbuild_raw<double>(c.stream, m, c.d_par.get(), xs::G_CIS, nvec, R, G, nullptr, scratch,
                           scratch + static_cast<size_t>(m.np) * nvec);
    return XS_OK;
  } catch (const xs::Error& e) {
    c.err = e.what();
    return e.status;
  } catch (const std::exception& e) {
    c.err = e.what();
    return XS_ECUDA;
  }
}
