// Learned Davidson guess and diagonal preconditioner of libxs (mlp.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace xs {

constexpr int kMlpFeatures = 11;
constexpr int kMlpHidden = 256;
constexpr int kMlpLayers = 4;
constexpr int kMlpOutputs = 2;   // 0: diagonal shift (eV), 1: log10 pair weight

// TF32 operand pairs and error word of the layers' tensor-core products (split
// TF32, float32 accumulation).  The caller keeps one per stream in its
// persistent workspace, so repeated network passes allocate nothing.
struct MlpOperands {
  DevBuf<float> ah, al, bh, bl;
  DevBuf<int> err;   // set by a timed-out bounded device wait
};

struct Mlp {
  int sizes[kMlpLayers + 1] = {kMlpFeatures, kMlpHidden, kMlpHidden, kMlpHidden, kMlpOutputs};
  DevBuf<float> w, wq, m, v, g;   // master weights, bfloat16-rounded copy, Adam moments, gradient
  int step = 0;
  bool ready = false;
  int nparams() const;
  void init(cudaStream_t s, unsigned long long seed);
  void set(cudaStream_t s, const float* host);
  void get(cudaStream_t s, float* host) const;
  void forward(cudaStream_t s, int rows, const float* X, std::vector<DevBuf<float>>& Z,
               std::vector<DevBuf<float>>& H, MlpOperands& mo) const;
  // gradient (into g) of the weighted mean-squared error with respect to the
  // parameters, evaluated with the bfloat16-rounded weights; returns the loss
  // (synchronises s and checks mo's error word)
  float gradient(cudaStream_t s, int rows, const float* X, const float* T, const float* colw, DevBuf<float>& scratch,
                 MlpOperands& mo);
  // one Adam step on the weighted mean-squared error; returns the loss
  float train_step(cudaStream_t s, int rows, const float* X, const float* T, const float* colw, float lr,
                   DevBuf<float>& scratch, MlpOperands& mo);
  // synchronises s, reads and clears mo's error word; throws XS_ETIMEOUT if it was set
  static void check(cudaStream_t s, MlpOperands& mo);
};

// indices i * nvir + a of the k lowest orbital-energy gaps eps[o + a] - eps[i],
// ascending (ties: lower index first)
std::vector<long long> lowest_gaps(const std::vector<double>& eps, int o, int v, long long k);
// the npairs lowest-gap pairs of a molecule (reads its orbital energies back)
std::vector<long long> lowest_gap_pairs(Ctx& c, const DevMol& m, int npairs);
// device scratch of pair_features, kept by the caller between calls
struct FeatureWork {
  DevBuf<double> stats, q, gam, t;
};
// features (npairs x kMlpFeatures, device) of the given pairs; dpairs receives
// the pair list on the device.  Asynchronous on the context's stream.
void pair_features(Ctx& c, const DevMol& m, const std::vector<long long>& pairs, float* F_dev,
                   DevBuf<long long>& dpairs, FeatureWork& fw);
// exact diagonal shift 2 (ia|ia) - (ii|aa) of the given pairs (device, float64)
void diagonal_shift(Ctx& c, const DevMol& m, const std::vector<long long>& pairs, double* shift_dev);

}  // namespace xs
