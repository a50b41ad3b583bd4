// Ground-state SCF of libxs (scf.cu).
#pragma once

#include "common.cuh"

namespace xs {

// Runs the closed-shell SCF of molecule m (integrals and core Hamiltonian
// already on the device); fills m.CT and m.eps.  Returns the iteration count.
int run_scf(Ctx& c, DevMol& m, double tol, int max_iter);
void destroy_solver(Ctx& c);

}  // namespace xs
