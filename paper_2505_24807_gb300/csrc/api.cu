// C ABI of libxs (declared and documented in include/xs.h).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "batch.h"
#include "davidson.h"
#include "mlp.h"
#include "ozaki.h"
#include "kernels.h"
#include "products.h"
#include "scf.h"
#include "syev.h"

using xs::Ctx;
using xs::DevBuf;
using xs::DevMol;
using xs::Error;

namespace {

template <typename F>
int guarded(xs_ctx* ctx, F&& f) {
  if (!ctx) return XS_EINVAL;
  ctx->c.err.clear();
  struct Bind {
    Bind(xs::Profiler* p) { xs::g_prof = p; }
    ~Bind() { xs::g_prof = nullptr; }
  } bind(&ctx->c.prof);
  try {
    XS_CUDA(cudaSetDevice(ctx->c.device));
    return f(ctx->c);
  } catch (const Error& e) {
    ctx->c.err = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    ctx->c.err = "host allocation failed";
    return XS_ENOMEM;
  } catch (const std::exception& e) {
    ctx->c.err = e.what();
    return XS_ECUDA;
  }
}

DevMol& molecule(Ctx& c, int mol) {
  if (mol < 0 || mol >= static_cast<int>(c.mols.size())) throw Error(XS_EINVAL, "molecule index out of range");
  DevMol& m = c.mols[mol];
  if (!m.ready) throw Error(XS_ESTATE, "molecule has no ground state");
  return m;
}

template <typename T>
void upload(cudaStream_t s, DevBuf<T>& d, const std::vector<T>& h) {
  d.alloc(h.size());
  if (!h.empty()) XS_CUDA(cudaMemcpyAsync(d.get(), h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
}

// copy count elements between host or device memory (unified addressing)
void copy_any(cudaStream_t s, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return;
  XS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

// A worker context for batched solves: the parent's parameters, its own
// non-blocking stream and scratch buffers.
std::unique_ptr<Ctx> make_worker(const Ctx& parent) {
  std::unique_ptr<Ctx> w(new Ctx());
  w->device = parent.device;
  for (int e = 0; e < XS_NELEM; ++e) w->par[e] = parent.par[e];
  w->have_params = true;
  XS_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
  w->own_stream = true;
  w->d_par.alloc(parent.d_par.n);
  XS_CUDA(cudaMemcpyAsync(w->d_par.get(), parent.d_par.get(), sizeof(double) * parent.d_par.n,
                          cudaMemcpyDeviceToDevice, w->stream));
  XS_CUDA(cudaStreamSynchronize(w->stream));
  return w;
}

void invalidate_mixed(DevMol& m) {
  m.dip.release();
  m.CTf_hi.release();
  m.CTf_lo.release();
  m.CTf.release();
}

}  // namespace

extern "C" {

int xs_create(xs_ctx** out, int device, void* stream) {
  if (!out) return XS_EINVAL;
  *out = nullptr;
  xs_ctx* ctx = nullptr;
  try {
    ctx = new xs_ctx();
  } catch (...) {
    return XS_ENOMEM;
  }
  ctx->c.device = device;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    delete ctx;
    return XS_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return XS_ECUDA;
  }
  if (stream) {
    ctx->c.stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->c.stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return XS_ECUDA;
    }
    ctx->c.own_stream = true;
  }
  *out = ctx;
  return XS_OK;
}

int xs_destroy(xs_ctx* ctx) {
  if (!ctx) return XS_OK;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  xs::destroy_solver(ctx->c);
  ctx->c.mols.clear();
  if (ctx->c.own_stream) cudaStreamDestroy(ctx->c.stream);
  delete ctx;
  return XS_OK;
}

const char* xs_last_error(const xs_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->c.err.c_str();
}

int xs_set_params(xs_ctx* ctx, const double* table, int n_elem) {
  return guarded(ctx, [&](Ctx& c) {
    if (!table || n_elem != XS_NELEM) throw Error(XS_EINVAL, "parameter table must have 4 rows (H, C, N, O)");
    std::vector<double> t(table, table + XS_NELEM * XS_NPARAM);
    for (int e = 0; e < XS_NELEM; ++e) {
      const double* r = table + e * XS_NPARAM;
      c.par[e] = xs::ElemParams{r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9], r[10], r[11], r[12]};
      if (!(r[4] > 0.0)) throw Error(XS_EINVAL, "gss must be positive");
    }
    upload(c.stream, c.d_par, t);
    XS_CUDA(cudaStreamSynchronize(c.stream));
    c.have_params = true;
    return XS_OK;
  });
}

int xs_ground_state(xs_ctx* ctx, int n_mol, const int* natoms, const int* Z, const double* xyz, double scf_tol,
                    int max_iter, xs_gs_info* info) {
  return guarded(ctx, [&](Ctx& c) {
    auto t0 = std::chrono::steady_clock::now();
    if (!c.have_params) throw Error(XS_ESTATE, "xs_set_params must come first");
    if (n_mol <= 0 || !natoms || !Z || !xyz) throw Error(XS_EINVAL, "bad molecule arrays");
    if (!(scf_tol > 0.0)) scf_tol = 1e-10;
    if (max_iter <= 0) max_iter = 300;
    cudaStream_t s = c.stream;
    c.mols.clear();
    c.mols.resize(n_mol);
    int off = 0, maxit = 0;
    for (int i = 0; i < n_mol; ++i) {
      DevMol& m = c.mols[i];
      if (natoms[i] <= 0) throw Error(XS_EINVAL, "molecule with no atoms");
      if (!xs::build_layout(natoms[i], Z + off, xyz + 3 * off, m.L))
        throw Error(XS_EINVAL, "molecule " + std::to_string(i) + ": odd electron count or unsupported element");
      off += natoms[i];
      m.n = m.L.nao;
      m.o = m.L.nocc;
      m.v = m.n - m.o;
      m.np = m.L.nprod;
      if (m.v <= 0) throw Error(XS_EINVAL, "no virtual orbitals");
      upload(s, m.ao_atom, m.L.ao_atom);
      upload(s, m.ao_local, m.L.ao_local);
      upload(s, m.atom_ao_off, m.L.ao_off);
      upload(s, m.atom_nao, m.L.nao_atom);
      upload(s, m.atom_prod_off, m.L.prod_off);
      upload(s, m.atom_elem, m.L.elem);
      upload(s, m.xyz, m.L.xyz);
      xs::build_model(s, m, c.d_par.get());   // two-centre supermatrix and core Hamiltonian
      xs::build_gtiles(s, m);
      xs::build_gpairs(s, m);
      int it = xs::run_scf(c, m, scf_tol, max_iter);
      maxit = it > maxit ? it : maxit;
      m.ready = true;
    }
    if (info) {
      info->n_mol = n_mol;
      info->max_scf_iter_used = maxit;
      info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return XS_OK;
  });
}

int xs_get_sizes(const xs_ctx* cctx, int mol, int* nao, int* nocc, int* natoms) {
  xs_ctx* ctx = const_cast<xs_ctx*>(cctx);
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (nao) *nao = m.n;
    if (nocc) *nocc = m.o;
    if (natoms) *natoms = m.L.natoms;
    return XS_OK;
  });
}

int xs_get_model(const xs_ctx* cctx, int mol, double* W, double* H, int* nprod) {
  xs_ctx* ctx = const_cast<xs_ctx*>(cctx);
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (nprod) *nprod = m.np;
    if (W) copy_any(c.stream, W, m.W.get(), sizeof(double) * m.np * m.np);
    if (H) copy_any(c.stream, H, m.H.get(), sizeof(double) * m.n * m.n);
    XS_CUDA(cudaStreamSynchronize(c.stream));
    return XS_OK;
  });
}

int xs_get_orbitals(const xs_ctx* cctx, int mol, double* C, double* eps) {
  xs_ctx* ctx = const_cast<xs_ctx*>(cctx);
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    const size_t nn = (size_t)m.n * m.n;
    if (C) {
      DevBuf<double> t(nn);
      xs::transpose(c.stream, m.n, m.n, m.CT.get(), t.get());
      copy_any(c.stream, C, t.get(), nn * sizeof(double));
      XS_CUDA(cudaStreamSynchronize(c.stream));
    }
    if (eps) copy_any(c.stream, eps, m.eps.get(), m.n * sizeof(double));
    XS_CUDA(cudaStreamSynchronize(c.stream));
    return XS_OK;
  });
}

int xs_set_orbitals(xs_ctx* ctx, int mol, const double* C, const double* eps) {
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (!C || !eps) throw Error(XS_EINVAL, "C and eps are required");
    const size_t nn = (size_t)m.n * m.n;
    DevBuf<double> t(nn);
    copy_any(c.stream, t.get(), C, nn * sizeof(double));
    xs::transpose(c.stream, m.n, m.n, t.get(), m.CT.get());
    copy_any(c.stream, m.eps.get(), eps, m.n * sizeof(double));
    XS_CUDA(cudaStreamSynchronize(c.stream));
    invalidate_mixed(m);
    return XS_OK;
  });
}

int xs_apply(xs_ctx* ctx, int mol, int kind, int nvec, const double* in, double* out, int precision) {
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (nvec < 0 || (nvec > 0 && (!in || !out))) throw Error(XS_EINVAL, "bad vectors");
    if (precision != XS_FP64 && precision != XS_MIXED) throw Error(XS_EINVAL, "bad precision");
    if (nvec == 0) return XS_OK;
    cudaStream_t s = c.stream;
    const long long ov = (long long)m.o * m.v, nn = (long long)m.n * m.n;
    if (kind == XS_KIND_G) {
      DevBuf<double> R((size_t)nvec * nn), G((size_t)nvec * nn);
      copy_any(s, R.get(), in, sizeof(double) * nvec * nn);
      xs::gmatrix(c, m, precision, nvec, R.get(), G.get());
      copy_any(s, out, G.get(), sizeof(double) * nvec * nn);
    } else if (kind == XS_KIND_A || kind == XS_KIND_APB || kind == XS_KIND_AMB || kind == XS_KIND_A_TRIPLET ||
               kind == XS_KIND_APB_TRIPLET) {
      const bool triplet = kind == XS_KIND_A_TRIPLET || kind == XS_KIND_APB_TRIPLET;
      DevBuf<double> X((size_t)nvec * ov), Y1((size_t)nvec * ov), Y2;
      copy_any(s, X.get(), in, sizeof(double) * nvec * ov);
      if (kind == XS_KIND_A || kind == XS_KIND_A_TRIPLET) {
        xs::products(c, m, XS_CIS, precision, nvec, X.get(), Y1.get(), nullptr, triplet);
        xs::check_device_error(c);
        copy_any(s, out, Y1.get(), sizeof(double) * nvec * ov);
      } else {
        Y2.alloc((size_t)nvec * ov);
        xs::products(c, m, XS_TDHF, precision, nvec, X.get(), Y1.get(), Y2.get(), triplet);
        xs::check_device_error(c);
        copy_any(s, out, (kind == XS_KIND_AMB ? Y2 : Y1).get(), sizeof(double) * nvec * ov);
      }
    } else {
      throw Error(XS_EINVAL, "unknown product kind");
    }
    XS_CUDA(cudaStreamSynchronize(s));
    return XS_OK;
  });
}

int xs_excited(xs_ctx* ctx, const xs_ex_opts* opts, double* omega, double* osc, int* iters, double* resid,
               xs_solve_info* info) {
  return guarded(ctx, [&](Ctx& c) {
    auto t0 = std::chrono::steady_clock::now();
    if (!opts) throw Error(XS_EINVAL, "options required");
    xs_ex_opts o = *opts;
    if (o.method != XS_CIS && o.method != XS_TDHF) throw Error(XS_EINVAL, "method must be XS_CIS or XS_TDHF");
    if (o.nroots < 1) throw Error(XS_EINVAL, "nroots must be >= 1");
    if (!(o.tol > 0.0)) throw Error(XS_EINVAL, "tol must be positive");
    if (o.precision != XS_FP64 && o.precision != XS_MIXED) throw Error(XS_EINVAL, "bad precision");
    if (o.subspace < XS_SUBSPACE_AUTO || o.subspace > XS_SUBSPACE_EMULATED)
      throw Error(XS_EINVAL, "bad subspace option");
    if (o.spin != XS_SINGLET && o.spin != XS_TRIPLET) throw Error(XS_EINVAL, "spin must be XS_SINGLET or XS_TRIPLET");
    if (!(o.memory_limit >= 0.0)) throw Error(XS_EINVAL, "memory_limit must be >= 0");
    if (c.mols.empty()) throw Error(XS_ESTATE, "xs_ground_state must come first");
    const int K = o.nroots;
    int status = XS_OK;
    xs_solve_info inf{};
    inf.converged = 1;
    double tprod = 0.0;
    const int nmol = static_cast<int>(c.mols.size());
    std::vector<xs::SolveStats> stats(nmol);
    std::vector<int> rcs(nmol, XS_OK);
    if (o.batched < 0 || o.batched > 2) throw Error(XS_EINVAL, "batched must be 0, 1 or 2");
    const int form = o.batched;
    if (form == 1) {
      long long replays = 0;
      xs::davidson_batched(c, o, stats, rcs, &replays);
      inf.graph_launches = replays;
    } else if (form == 2 && nmol > 1) {
      // molecules advance concurrently: one host thread per worker context,
      // each launching on its own stream; the GPU overlaps their kernels
      unsigned hw = std::thread::hardware_concurrency();
      const int nw = std::max(1, std::min<int>(nmol, std::min<int>(hw ? static_cast<int>(hw) : 8, 16)));
      while (static_cast<int>(c.workers.size()) < nw) c.workers.push_back(make_worker(c));
      for (auto& wk : c.workers) wk->mlp = c.mlp;
      XS_CUDA(cudaStreamSynchronize(c.stream));
      std::atomic<int> next{0};
      std::vector<std::string> errs(nmol);
      std::vector<std::thread> th;
      for (int t = 0; t < nw; ++t) {
        th.emplace_back([&, t]() {
          cudaSetDevice(c.device);
          Ctx& w = *c.workers[t];
          for (int i = next++; i < nmol; i = next++) {
            try {
              rcs[i] = xs::davidson(w, c.mols[i], o, stats[i]);
            } catch (const Error& e) {
              rcs[i] = e.status;
              errs[i] = e.what();
            } catch (const std::exception& e) {
              rcs[i] = XS_ECUDA;
              errs[i] = e.what();
            }
          }
          cudaStreamSynchronize(w.stream);
        });
      }
      for (auto& x : th) x.join();
      for (int i = 0; i < nmol; ++i)
        if (!errs[i].empty()) throw Error(rcs[i], "molecule " + std::to_string(i) + ": " + errs[i]);
    } else {
      for (int i = 0; i < nmol; ++i) {
        molecule(c, i);
        rcs[i] = xs::davidson(c, c.mols[i], o, stats[i]);
      }
    }
    for (int ii = 0; ii < nmol; ++ii) {
      const size_t i = static_cast<size_t>(ii);
      DevMol& m = molecule(c, ii);
      xs::SolveStats& st = stats[ii];
      int rc = rcs[ii];
      if (rc == XS_EUNSTABLE) throw Error(XS_EUNSTABLE, "A - B is not positive definite (molecule " +
                                                            std::to_string(i) + ")");
      if (rc != XS_OK) status = rc;
      inf.iterations = st.iterations > inf.iterations ? st.iterations : inf.iterations;
      inf.products += st.products;
      inf.converged = inf.converged && st.converged;
      inf.polished = inf.polished || st.polished;
      inf.learned = inf.learned || st.learned;
      inf.fallback = inf.fallback || st.fallback;
      inf.max_subspace_used = st.smax > inf.max_subspace_used ? st.smax : inf.max_subspace_used;
      inf.tol_used = st.tol_used > inf.tol_used ? st.tol_used : inf.tol_used;
      tprod += st.seconds_products;
      const int kk = m.nroots;
      std::vector<double> pad(K, 0.0);
      auto put = [&](double* dst, const std::vector<double>& src) {
        if (!dst) return;
        std::vector<double> t(K, 0.0);
        for (int j = 0; j < kk && j < K; ++j) t[j] = src[j];
        copy_any(c.stream, dst + i * K, t.data(), sizeof(double) * K);
        XS_CUDA(cudaStreamSynchronize(c.stream));
      };
      put(omega, m.omega);
      put(osc, m.osc);
      put(resid, m.resid);
      if (iters) {
        int itv = m.iterations;
        copy_any(c.stream, iters + i, &itv, sizeof(int));
        XS_CUDA(cudaStreamSynchronize(c.stream));
      }
    }
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inf.seconds_products = tprod;
    if (info) *info = inf;
    if (status == XS_ENOCONV) c.err = "Davidson did not converge within max_iter";
    return status;
  });
}

int xs_gradient(xs_ctx* ctx, int mol, int root, double* grad, int* cg_iterations) {
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (m.nroots <= 0 || m.spin != XS_SINGLET || !m.U.get())
      throw Error(XS_ESTATE, "xs_gradient needs a singlet CIS or TDHF solution of the molecule");
    if (root < 0 || root >= m.nroots) throw Error(XS_EINVAL, "root out of range");
    if (!grad) throw Error(XS_EINVAL, "null gradient array");
    std::vector<double> g((size_t)XS_NELEM * XS_NPARAM);
    int its = 0;
    xs::parameter_gradient(c, m, root, g.data(), &its);
    copy_any(c.stream, grad, g.data(), sizeof(double) * g.size());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    if (cg_iterations) *cg_iterations = its;
    return XS_OK;
  });
}

int xs_spectrum(xs_ctx* ctx, int n, const double* omega, const double* f, double width, int ngrid,
                const double* grid, double* out) {
  return guarded(ctx, [&](Ctx& c) {
    if (n < 0 || ngrid < 0) throw Error(XS_EINVAL, "negative count");
    if (!(width > 0.0) || !std::isfinite(width)) throw Error(XS_EINVAL, "width must be positive and finite");
    if ((n > 0 && (!omega || !f)) || (ngrid > 0 && (!grid || !out))) throw Error(XS_EINVAL, "null array");
    if (ngrid == 0) return XS_OK;
    cudaStream_t s = c.stream;
    DevBuf<double> buf((size_t)2 * n + 2 * (size_t)ngrid);
    double* dw = buf.get();
    double* df = dw + n;
    double* dg = df + n;
    double* dout = dg + ngrid;
    if (n > 0) {
      copy_any(s, dw, omega, sizeof(double) * n);
      copy_any(s, df, f, sizeof(double) * n);
    }
    copy_any(s, dg, grid, sizeof(double) * ngrid);
    xs::absorption_spectrum(s, n, dw, df, width, ngrid, dg, dout);
    copy_any(s, out, dout, sizeof(double) * ngrid);
    XS_CUDA(cudaStreamSynchronize(s));
    return XS_OK;
  });
}

int xs_get_amplitudes(const xs_ctx* cctx, int mol, int root, double* X, double* Y, size_t ov) {
  xs_ctx* ctx = const_cast<xs_ctx*>(cctx);
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (m.nroots == 0) throw Error(XS_ESTATE, "no excited-state solution");
    if (root < 0 || root >= m.nroots) throw Error(XS_EINVAL, "root out of range");
    const long long n_ov = (long long)m.o * m.v;
    if ((long long)ov != n_ov) throw Error(XS_EINVAL, "ov must equal nocc * nvir");
    cudaStream_t s = c.stream;
    DevBuf<double> t((size_t)n_ov);
    const double* U = m.U.get() + root * n_ov;
    const double* W = m.Wv.get() + root * n_ov;
    if (X) {
      // X = (U + W) / 2
      XS_CUDA(cudaMemcpyAsync(t.get(), U, sizeof(double) * n_ov, cudaMemcpyDeviceToDevice, s));
      xs::axpy(s, n_ov, 1.0, W, t.get());
      xs::scal(s, n_ov, 0.5, t.get());
      copy_any(s, X, t.get(), sizeof(double) * n_ov);
      XS_CUDA(cudaStreamSynchronize(s));
    }
    if (Y) {
      XS_CUDA(cudaMemcpyAsync(t.get(), U, sizeof(double) * n_ov, cudaMemcpyDeviceToDevice, s));
      xs::axpy(s, n_ov, -1.0, W, t.get());
      xs::scal(s, n_ov, 0.5, t.get());
      copy_any(s, Y, t.get(), sizeof(double) * n_ov);
      XS_CUDA(cudaStreamSynchronize(s));
    }
    return XS_OK;
  });
}

int xs_mlp_nparams(void) {
  xs::Mlp m;
  return m.nparams();
}

int xs_mlp_init(xs_ctx* ctx, unsigned long long seed) {
  return guarded(ctx, [&](Ctx& c) {
    if (!c.mlp) c.mlp = std::make_shared<xs::Mlp>();
    c.mlp->init(c.stream, seed);
    XS_CUDA(cudaStreamSynchronize(c.stream));
    return XS_OK;
  });
}

int xs_mlp_get_weights(xs_ctx* ctx, float* w) {
  return guarded(ctx, [&](Ctx& c) {
    if (!c.mlp || !c.mlp->ready) throw Error(XS_ESTATE, "no network");
    if (!w) throw Error(XS_EINVAL, "null buffer");
    std::vector<float> h(c.mlp->nparams());
    c.mlp->get(c.stream, h.data());
    copy_any(c.stream, w, h.data(), sizeof(float) * h.size());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    return XS_OK;
  });
}

int xs_mlp_set_weights(xs_ctx* ctx, const float* w) {
  return guarded(ctx, [&](Ctx& c) {
    if (!w) throw Error(XS_EINVAL, "null buffer");
    if (!c.mlp) c.mlp = std::make_shared<xs::Mlp>();
    std::vector<float> h(c.mlp->nparams());
    copy_any(c.stream, h.data(), w, sizeof(float) * h.size());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    c.mlp->set(c.stream, h.data());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    return XS_OK;
  });
}

int xs_mlp_features(xs_ctx* ctx, int mol, int npairs, float* features, long long* pairs, int* count) {
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (npairs <= 0 || !features) throw Error(XS_EINVAL, "bad request");
    std::vector<long long> pr = xs::lowest_gap_pairs(c, m, npairs);
    DevBuf<float> F(pr.size() * xs::kMlpFeatures);
    DevBuf<long long> dp;
    xs::FeatureWork fw;
    xs::pair_features(c, m, pr, F.get(), dp, fw);
    copy_any(c.stream, features, F.get(), sizeof(float) * F.n);
    if (pairs) copy_any(c.stream, pairs, pr.data(), sizeof(long long) * pr.size());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    if (count) *count = static_cast<int>(pr.size());
    return XS_OK;
  });
}

int xs_mlp_targets(xs_ctx* ctx, int mol, int npairs, const long long* pairs, float* targets) {
  return guarded(ctx, [&](Ctx& c) {
    DevMol& m = molecule(c, mol);
    if (npairs <= 0 || !pairs || !targets) throw Error(XS_EINVAL, "bad request");
    if (m.nroots == 0) throw Error(XS_ESTATE, "solve the molecule first (amplitudes give the weight targets)");
    std::vector<long long> pr(npairs);
    copy_any(c.stream, pr.data(), pairs, sizeof(long long) * npairs);
    XS_CUDA(cudaStreamSynchronize(c.stream));
    const long long ov = (long long)m.o * m.v;
    for (long long p : pr)
      if (p < 0 || p >= ov) throw Error(XS_EINVAL, "pair index out of range");
    DevBuf<double> sh(npairs);
    xs::diagonal_shift(c, m, pr, sh.get());
    std::vector<double> shh(npairs);
    XS_CUDA(cudaMemcpyAsync(shh.data(), sh.get(), sizeof(double) * npairs, cudaMemcpyDeviceToHost, c.stream));
    // weight of each pair in the stored roots (X+Y for TDHF, X for CIS)
    std::vector<double> U((size_t)m.nroots * ov);
    XS_CUDA(cudaMemcpyAsync(U.data(), m.U.get(), sizeof(double) * U.size(), cudaMemcpyDeviceToHost, c.stream));
    XS_CUDA(cudaStreamSynchronize(c.stream));
    std::vector<float> t((size_t)npairs * 2);
    for (int q = 0; q < npairs; ++q) {
      double wgt = 0.0;
      for (int r = 0; r < m.nroots; ++r) {
        const double u = U[(size_t)r * ov + pr[q]];
        wgt += u * u;
      }
      t[2 * q] = static_cast<float>(shh[q]);
      t[2 * q + 1] = static_cast<float>(std::log10(std::max(wgt, 1e-6)));
    }
    copy_any(c.stream, targets, t.data(), sizeof(float) * t.size());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    return XS_OK;
  });
}

int xs_mlp_forward(xs_ctx* ctx, int rows, const float* features, float* out) {
  return guarded(ctx, [&](Ctx& c) {
    if (!c.mlp || !c.mlp->ready) throw Error(XS_ESTATE, "no network");
    if (rows <= 0 || !features || !out) throw Error(XS_EINVAL, "bad request");
    DevBuf<float> F((size_t)rows * xs::kMlpFeatures);
    copy_any(c.stream, F.get(), features, sizeof(float) * F.n);
    std::vector<DevBuf<float>> Z, H;
    xs::MlpOperands mo;
    c.mlp->forward(c.stream, rows, F.get(), Z, H, mo);
    copy_any(c.stream, out, H[xs::kMlpLayers - 1].get(), sizeof(float) * rows * xs::kMlpOutputs);
    xs::Mlp::check(c.stream, mo);
    return XS_OK;
  });
}

int xs_mlp_grad(xs_ctx* ctx, int rows, const float* features, const float* targets, float* grad, float* loss) {
  return guarded(ctx, [&](Ctx& c) {
    if (!c.mlp || !c.mlp->ready) throw Error(XS_ESTATE, "initialise or load the network first");
    if (rows <= 0 || !features || !targets || !grad) throw Error(XS_EINVAL, "bad request");
    DevBuf<float> F((size_t)rows * xs::kMlpFeatures), T((size_t)rows * xs::kMlpOutputs), colw(2), scratch;
    copy_any(c.stream, F.get(), features, sizeof(float) * F.n);
    copy_any(c.stream, T.get(), targets, sizeof(float) * T.n);
    const float cw[2] = {0.01f, 1.0f};
    copy_any(c.stream, colw.get(), cw, sizeof(cw));
    xs::MlpOperands mo;
    const float l = c.mlp->gradient(c.stream, rows, F.get(), T.get(), colw.get(), scratch, mo);
    copy_any(c.stream, grad, c.mlp->g.get(), sizeof(float) * c.mlp->nparams());
    XS_CUDA(cudaStreamSynchronize(c.stream));
    if (loss) *loss = l;
    return XS_OK;
  });
}

int xs_mlp_train(xs_ctx* ctx, int rows, const float* features, const float* targets, int epochs, int batch,
                 float lr, float* loss) {
  return guarded(ctx, [&](Ctx& c) {
    if (!c.mlp || !c.mlp->ready) throw Error(XS_ESTATE, "initialise or load the network first");
    if (rows <= 0 || epochs <= 0 || batch <= 0 || !features || !targets) throw Error(XS_EINVAL, "bad request");
    DevBuf<float> F((size_t)rows * xs::kMlpFeatures), T((size_t)rows * xs::kMlpOutputs), colw(2), scratch;
    copy_any(c.stream, F.get(), features, sizeof(float) * F.n);
    copy_any(c.stream, T.get(), targets, sizeof(float) * T.n);
    const float cw[2] = {0.01f, 1.0f};
    copy_any(c.stream, colw.get(), cw, sizeof(cw));
    XS_CUDA(cudaStreamSynchronize(c.stream));
    xs::MlpOperands mo;
    for (int e = 0; e < epochs; ++e) {
      double sum = 0.0;
      int nb = 0;
      for (int r0 = 0; r0 < rows; r0 += batch) {
        const int rb = std::min(batch, rows - r0);
        sum += c.mlp->train_step(c.stream, rb, F.get() + (size_t)r0 * xs::kMlpFeatures,
                                 T.get() + (size_t)r0 * xs::kMlpOutputs, colw.get(), lr, scratch, mo);
        ++nb;
      }
      if (loss) loss[e] = static_cast<float>(sum / nb);
    }
    return XS_OK;
  });
}

int xs_profile(xs_ctx* ctx, int enable) {
  return guarded(ctx, [&](Ctx& c) {
    if (enable < 0 || enable > 3) throw Error(XS_EINVAL, "xs_profile: enable must be 0, 1, 2 or 3");
    c.prof.reset();
    c.prof.on = enable != 0;
    c.prof.events = enable == 1 || enable == 3;
    c.prof.timeline = enable == 3;
    return XS_OK;
  });
}

int xs_profile_read(xs_ctx* ctx, xs_prof_entry* out, int max_entries, int* count) {
  return guarded(ctx, [&](Ctx& c) {
    XS_CUDA(cudaStreamSynchronize(c.stream));
    c.prof.flush();
    int k = 0;
    for (auto& kv : c.prof.e) {
      if (out && k < max_entries) {
        xs_prof_entry& e = out[k];
        std::memset(&e, 0, sizeof(e));
        std::strncpy(e.name, kv.first.c_str(), sizeof(e.name) - 1);
        e.launches = kv.second.launches;
        e.ms = kv.second.ms;
        e.bytes = kv.second.bytes;
        e.flops = kv.second.flops;
      }
      ++k;
    }
    // one more entry: every library kernel launch while profiling was on
    if (out && k < max_entries) {
      xs_prof_entry& e = out[k];
      std::memset(&e, 0, sizeof(e));
      std::strncpy(e.name, "all_launches", sizeof(e.name) - 1);
      e.launches = static_cast<int>(c.prof.launches);
    }
    ++k;
    if (count) *count = k;
    return XS_OK;
  });
}

int xs_subspace_gram(xs_ctx* ctx, int M, int N, long long L, const double* A, const double* B, double* C,
                     int emulated) {
  return guarded(ctx, [&](Ctx& c) {
    if (M < 0 || N < 0 || L < 1 || (M > 0 && N > 0 && (!A || !B || !C)))
      throw Error(XS_EINVAL, "bad gram arguments");
    if (M == 0 || N == 0) return XS_OK;
    if (L > (1LL << 31) - 1024) throw Error(XS_EINVAL, "vectors too long");
    cudaStream_t s = c.stream;
    DevBuf<double> dA((size_t)M * L), dB((size_t)N * L), dC((size_t)M * N);
    copy_any(s, dA.get(), A, sizeof(double) * M * L);
    copy_any(s, dB.get(), B, sizeof(double) * N * L);
    if (emulated) {
      if (!c.tc_err.get()) {
        c.tc_err.alloc(1);
        XS_CUDA(cudaMemsetAsync(c.tc_err.get(), 0, sizeof(int), s));
      }
      const long long Lp = xs::oz_lp(L);
      DevBuf<xs::oz_t> ta((size_t)M * xs::kOzDigits * Lp), tb((size_t)N * xs::kOzDigits * Lp);
      DevBuf<int> eA(M), eB(N);
      xs::OzWork w;
      xs::oz_exponents(s, M, L, dA.get(), L, eA.get(), w, c.tc_err.get());
      xs::oz_exponents(s, N, L, dB.get(), L, eB.get(), w, c.tc_err.get());
      const long long PA = (long long)M * xs::kOzDigits, PB = (long long)N * xs::kOzDigits;   // plane capacities
      xs::oz_slice(s, M, L, dA.get(), L, eA.get(), ta.get(), PA, 0, nullptr, 0, 0);
      xs::oz_slice(s, N, L, dB.get(), L, eB.get(), tb.get(), PB, 0, nullptr, 0, 0);
      xs::oz_gram(s, M, N, L, ta.get(), PA, eA.get(), tb.get(), PB, eB.get(), 1.0, 0.0, dC.get(), N, w,
                  c.tc_err.get());
      xs::check_device_error(c);
    } else {
      xs::gram<double>(s, M, N, static_cast<int>(L), dA.get(), static_cast<int>(L), dB.get(), static_cast<int>(L),
                       dC.get(), N, 1.0, 0.0, c.ws0);
    }
    copy_any(s, C, dC.get(), sizeof(double) * M * N);
    XS_CUDA(cudaStreamSynchronize(s));
    return XS_OK;
  });
}

int xs_subspace_eig(xs_ctx* ctx, int S, int k, const double* A, double* w, double* Z) {
  return guarded(ctx, [&](Ctx& c) {
    if (S < 1 || S > 1024 || k < 1 || k > S || !A || !w || !Z) throw Error(XS_EINVAL, "bad eigensolver arguments");
    cudaStream_t s = c.stream;
    DevBuf<double> dA((size_t)S * S), dw((size_t)k), dZ((size_t)S * k), scratch;
    DevBuf<int> info(1);
    copy_any(s, dA.get(), A, sizeof(double) * S * S);
    xs::syevk(s, S, k, dA.get(), S, dw.get(), dZ.get(), k, scratch, info.get());
    copy_any(s, w, dw.get(), sizeof(double) * k);
    copy_any(s, Z, dZ.get(), sizeof(double) * S * k);
    XS_CUDA(cudaStreamSynchronize(s));
    return XS_OK;
  });
}

int xs_subspace_combine(xs_ctx* ctx, int nb, int S, int nout, long long L, const double* X, const double* coef,
                        double* Y, int emulated) {
  return guarded(ctx, [&](Ctx& c) {
    if (nb < 1 || nb > 3 || S < 1 || nout < 0 || L < 1 || (nout > 0 && (!X || !coef || !Y)))
      throw Error(XS_EINVAL, "bad combine arguments");
    if (nout == 0) return XS_OK;
    if (L > (1LL << 31) - 1024) throw Error(XS_EINVAL, "vectors too long");
    cudaStream_t s = c.stream;
    DevBuf<double> dX((size_t)nb * S * L), dc((size_t)nb * S * nout), dY((size_t)nout * L);
    copy_any(s, dX.get(), X, sizeof(double) * nb * S * L);
    copy_any(s, dc.get(), coef, sizeof(double) * nb * S * nout);
    if (emulated) {
      if (!c.tc_err.get()) {
        c.tc_err.alloc(1);
        XS_CUDA(cudaMemsetAsync(c.tc_err.get(), 0, sizeof(int), s));
      }
      const int ldk = xs::oz_ldk(S);
      DevBuf<xs::oz_t> nn((size_t)nb * L * ldk);
      // digit columns past S * 8 are read (times zero coefficients): clear them
      XS_CUDA(cudaMemsetAsync(nn.get(), 0, sizeof(xs::oz_t) * nb * L * ldk, s));
      DevBuf<int> e((size_t)nb * S);
      xs::OzWork w;
      xs::OzBlock blk[3];
      for (int b = 0; b < nb; ++b) {
        const double* Xb = dX.get() + (size_t)b * S * L;
        xs::oz_exponents(s, S, L, Xb, L, e.get() + b * S, w, c.tc_err.get());
        xs::oz_slice(s, S, L, Xb, L, e.get() + b * S, nullptr, 0, 0, nn.get() + (size_t)b * L * ldk, ldk, 0);
        blk[b] = xs::OzBlock{nn.get() + (size_t)b * L * ldk, ldk, e.get() + b * S, dc.get() + (size_t)b * S * nout,
                             nout};
      }
      xs::oz_combine(s, nb, blk, S, nout, L, 1.0, 0.0, dY.get(), L, w, c.tc_err.get());
      xs::check_device_error(c);
    } else {
      for (int b = 0; b < nb; ++b)
        xs::gemm<double>(s, true, false, nout, static_cast<int>(L), S, 1.0, dc.get() + (size_t)b * S * nout, nout, 0,
                         dX.get() + (size_t)b * S * L, static_cast<int>(L), 0, b == 0 ? 0.0 : 1.0, dY.get(),
                         static_cast<int>(L), 0, 1);
    }
    copy_any(s, Y, dY.get(), sizeof(double) * nout * L);
    XS_CUDA(cudaStreamSynchronize(s));
    return XS_OK;
  });
}

}  // extern "C"
