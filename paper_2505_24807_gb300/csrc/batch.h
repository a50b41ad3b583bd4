// Lock-step batched Davidson of libxs (batch.cu).
#pragma once

#include <vector>

#include "common.cuh"
#include "davidson.h"

namespace xs {

// Largest root count of the lock-step batched solver (its subspaces hold at
// most kBatchMaxSub vectors and its per-molecule small matrices live in shared
// memory).
constexpr int kBatchMaxRoots = 16;
constexpr int kBatchMaxSub = 128;
// Molecules per lock-step group: the ragged kernels' work-list prologue keeps
// one prefix entry per molecule in shared memory.
constexpr int kBatchGroup = 1024;

// Solves every molecule of c.mols together: one captured CUDA graph per
// Davidson iteration for the whole batch (see batch.cu).  Fills each
// molecule's roots, oscillator strengths, residuals and amplitudes like
// davidson() and returns per-molecule status codes in rcs (XS_OK,
// XS_ENOCONV, XS_EUNSTABLE).  graph_launches: graph replays made.
void davidson_batched(Ctx& c, const xs_ex_opts& opt, std::vector<SolveStats>& st, std::vector<int>& rcs,
                      long long* graph_launches);

}  // namespace xs
