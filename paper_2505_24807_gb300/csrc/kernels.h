// Host-side launchers of libxs's CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace xs {

// ---- dense algebra (gemm.cu) ------------------------------------------------
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], row-major storage; op(A) is M x K,
// op(B) is K x N.  transA: A is stored K x M; transB: B is stored N x K.
template <typename T>
void gemm(cudaStream_t s, bool transA, bool transB, int M, int N, int K, T alpha, const T* A,
          int lda, long long sA, const T* B, int ldb, long long sB, T beta, T* C, int ldc,
          long long sC, int batch = 1);

// While alive on a thread, GEMM calls skip the tile-shape autotuner (which
// allocates a scratch output and synchronises the stream on a new problem
// class): for allocation-free entry points.
struct NoTuneScope {
  NoTuneScope();
  ~NoTuneScope();
};
// True while a NoTuneScope is alive on this thread.
bool tuning_disabled();

// C (M x N) = alpha A (M x L) B(N x L)^T + beta C for long L (split over L).
template <typename T>
void gram(cudaStream_t s, int M, int N, int L, const T* A, int lda, const T* B, int ldb, T* C,
          int ldc, T alpha, T beta, DevBuf<T>& ws);

// ---- G(R) build (gbuild.cu) -------------------------------------------------
// G(R) variants: singlet CIS 2J(R) - K(R); singlet TDHF G+ = 4J(R_s) - 2K(R_s)
// with G- = -2K(R_a); triplets drop the Coulomb terms: CIS -K(R), TDHF
// G+ = -2K(R_s) with the same G- (A - B does not depend on the spin).
enum GMode { G_CIS = 0, G_RPA = 1, G_CIS_T = 2, G_RPA_T = 3 };
inline GMode gmode(bool rpa, bool triplet) {
  return rpa ? (triplet ? G_RPA_T : G_RPA) : (triplet ? G_CIS_T : G_CIS);
}
// nvec AO matrices R (n x n each, row-major, consecutive) -> G (CIS/Fock:
// 2J(R) - K(R)) or G+ = 4J(Rs) - 2K(Rs) and G- = -2K(Ra) (RPA).
// Gm is unused for G_CIS.  ws: scratch of at least 2 * np * nvec.
template <typename T>
void gbuild(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const T* R,
            T* G, T* Gm, DevBuf<T>& ws);
// Float32 G build whose output is the TF32 pair (hi, lo) of G (and G- for
// TDHF) with row stride ldo >= n (batch stride n * ldo, columns n..ldo-1
// zeroed): the back-transform's tensor-core operand without a separate split.
void gbuild_split(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* R,
                  float* Gh, float* Gl, float* Gmh, float* Gml, int ldo, DevBuf<float>& ws);
// Atom-aligned tiling of G used by gbuild (rows: one heavy atom or up to 4
// hydrogens; columns: whole atoms, at most 64 AOs); built once per molecule.
void build_gtiles(cudaStream_t s, DevMol& m);
// Two-centre product supermatrix m.W (np x np) and core Hamiltonian m.H
// (n x n) on the device from the uploaded layout and parameters (integrals.cu).
void build_model(cudaStream_t s, DevMol& m, const double* d_par);
// Super-atoms (a heavy atom, or up to 4 consecutive hydrogens) and their
// unordered pairs in warp blocks (gpair.cu); built once per molecule.
void build_gpairs(cudaStream_t s, DevMol& m);
// Float32 G build over super-atom pairs (gpair.cu): every R element read and
// every G element written once per matrix.  J2 (np x nvec, row stride ldj) is
// the two-centre Coulomb of the diagonal blocks.  Plain outputs with row
// stride n, or TF32 pairs with row stride ldo (split).
// J2 = W r for symmetric float32 W (np x np), r and J2 np x nvec (row stride
// nvec); ws: partial sums (grown as needed)
void coulomb_j2(cudaStream_t s, int np, int nvec, const float* W, const float* r, float* J2, DevBuf<float>& ws);
void gpair_build(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* W,
                 const float* J2, int ldj, const float* R, float* G, float* Gm);
void gpair_build_split(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const float* W,
                       const float* J2, int ldj, const float* R, float* Gh, float* Gl, float* Gmh, float* Gml,
                       int ldo);
// The same with caller-provided scratch: r and J2 of np * nvec elements each.
template <typename T>
void gbuild_raw(cudaStream_t s, const DevMol& m, const double* d_par, GMode mode, int nvec, const T* R, T* G,
                T* Gm, T* r, T* J2);

// ---- elementwise helpers (vec.cu) ---------------------------------------------
template <typename T>
void add_diag_term(cudaStream_t s, int nvec, int o, int v, const double* eps, const T* X, T* Y);
void precondition(cudaStream_t s, int nvec, int o, int v, const double* eps, const double* omega,
                  const double* R, double* T, const double* shift = nullptr);
void scatter(cudaStream_t s, int n, const long long* idx, const double* val, double* out);  // out[idx[k]] = val[k]
void residual_norms(cudaStream_t s, int nvec, long long len, const double* A, const double* B,
                    const double* omega, double* out_norm, double* R);
void row_norms(cudaStream_t s, int nvec, long long len, const double* X, double* out_norm);
// X[r] *= scale[r]; rowmax (optional, zeroed here): per row abs_hi
// (common.cuh) of the largest |scaled x|
void scale_rows(cudaStream_t s, int nvec, long long len, double* X, const double* scale,
                unsigned int* rowmax = nullptr);
void convert_d2f(cudaStream_t s, long long n, const double* a, float* b);
void convert_f2d(cudaStream_t s, long long n, const float* a, double* b);
void split_d2f(cudaStream_t s, long long n, const double* a, float* hi, float* lo);
void fill(cudaStream_t s, long long n, double* a, double v);
void axpy(cudaStream_t s, long long n, double alpha, const double* x, double* y);
void scal(cudaStream_t s, long long n, double alpha, double* x);
void max_abs(cudaStream_t s, long long n, const double* a, double* out);   // out: one device double
void transpose(cudaStream_t s, int rows, int cols, const double* a, double* b);
// Synchronise the context's stream and raise XS_ETIMEOUT (clearing the word)
// when a tensor-core kernel's bounded wait gave up or a digit split met a
// non-finite value (the error word c.tc_err).
void check_device_error(Ctx& c);

// ---- absorption spectrum (spectrum.cu) -----------------------------------
// out[g] = sum_n f_n exp(-(grid_g - omega_n)^2 / (2 width^2)) / (width sqrt(2 pi)),
// all arrays on the device.
void absorption_spectrum(cudaStream_t s, int n, const double* omega, const double* f, double width, int ngrid,
                         const double* grid, double* out);

// ---- small dense eigenproblems (small.cu) -----------------------------------
// Symmetric eigen-decomposition (n <= 1024) by cyclic Jacobi in one CTA
// (shared-memory resident for n <= 64): A (n x n, lda) may be overwritten, V
// gets the eigenvectors in columns (ldv), w the eigenvalues in ascending order.
void jacobi_eig(cudaStream_t s, int n, double* A, int lda, double* V, int ldv, double* w, int* info);

}  // namespace xs
