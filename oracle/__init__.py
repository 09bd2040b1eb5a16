"""FP64 CPU oracle for the finite-difference micromagnetic hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_1406_7635_gb300/csrc``); the only module
both sides read is ``paper_1406_7635_gb300/workloads.py``, which builds seeded
synthetic inputs and holds none of the method's arithmetic.

Everything here is plain numpy in float64, written to be checked against the
paper ("The design and verification of Mumax3", Vansteenkiste et al.) by eye:

* ``newell``  -- cell-averaged demagnetising tensor (Sec. III.B "Magnetostatic
  kernel"): Newell's analytic f/g integrals near the source, Gauss-Legendre
  integration of the point-dipole tensor far from it.
* ``demag``   -- the magnetostatic convolution B_demag = K * M (Sec. III.B),
  either by direct O(N^2) summation or by a zero-padded FFT (numpy's FFT as a
  library primitive).
* ``field``   -- exchange (Eqs. for B_exch incl. the inter-region harmonic
  mean), uniaxial anisotropy, Zeeman, effective field, Landau-Lifshitz torque
  (Eq. eqLLG).
* ``dmi``     -- interfacial Dzyaloshinskii-Moriya field and its boundary
  conditions (Sec. III).
* ``stt``     -- Zhang-Li and Slonczewski spin-transfer torques (Sec. III).
* ``rk45``    -- Dormand-Prince RK45 with the adaptive step control of Sec. IV.
* ``relax``   -- Bogacki-Shampine RK23 and relax() (Sec. IV).
* ``fno``     -- the Fourier-neural-operator surrogate of the demag field
  (forward and backward; the paper has none).
* ``energy``  -- energies from the effective field (Eqs. for E_demag, E_exch,
  E_anis).

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, a printed table value of the
paper, an invariant or a brute-force evaluation.  One reading is unpinned:
trajectory agreement of chaotic switching beyond a replayed step sequence
("parity unpinned" for free-running adaptive trajectories; only statistics are
compared there).
"""
