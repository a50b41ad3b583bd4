"""Plain FP64 CPU oracle for the semiempirical CIS / TDHF excited-state method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It follows arXiv:2505.24807 ("PySEQM 2.0", Section "Theory and
implementation"):

* ``nddo``     -- the synthetic NDDO model: one-centre parameters, two-centre
                  multipole integrals, overlap and core Hamiltonian, dipoles.
* ``scf``      -- Coulomb / exchange builds and the restricted closed-shell
                  SCF, F C = C eps with S = I (Eq. 1).
* ``excited``  -- explicit A and B (Eq. A_matrix_elem), brute-force CIS and
                  RPA (Eqs. rpa_eqn, cis_eqn), the A*V product through the AO
                  transition density (Eqs. cis_matrix_vector, ftilde), block
                  Davidson for CIS and for RPA, oscillator strengths, and the
                  spin-adapted triplet forms (beyond the paper's singlets).
* ``spectrum`` -- the absorption spectrum: oscillator strengths broadened by
                  Gaussians (Section "Results and discussion").
* ``mlp``      -- the learned guess network's forward and backward pass.

Everything is float64, written for clarity rather than speed.  Where the
paper is silent (spin adaptation, the NDDO parameters and integral formulas,
the RPA Davidson variant, guesses and thresholds) the reading taken is stated
at the function that implements it.

Parity status: every function is pinned by a test under ``tests/`` against
brute force, closed forms or invariants, except absolute excitation energies
of real molecules with real AM1 parameters, which are "parity unpinned"
because the paper prints neither the parameters nor per-molecule values.
"""
