"""FP64 CPU oracle for the Mera state-vector path (arXiv 2411.15332).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference arm of ``bench.py`` may import this package.
The CUDA library never calls it, and it shares no code with the CUDA
library: the two sides meet only through the seeded input generators in
``paper_2411_15332_gb300.inputs``, which hold no simulation arithmetic.

Everything is plain numpy in float64 / complex128, slow and literal:

* ``gates``       gate matrices of the paper's gate survey (Table I).
* ``statevector`` the operation matrix by the literal MTP (Eq. 6) and the
                  MVM (Eq. 7) for n <= 10; per-gate tensor-axis application
                  for any n; readouts (Eq. 4-5).
* ``dax``         the DAX and DAS compressed structures, their MTP and MVM
                  (Sec. III-A).
* ``rh``          the RH structure of H^{(x)n}, its sign rule and the four
                  MVM methods with sign-computation counters (Sec. III-B,
                  Table II, Algorithm 1).
* ``circuits``    applies gate lists, traces single amplitudes of monomial
                  circuits, QNN forward and parameter-shift / finite
                  difference gradients, Grover closed form.

Parity status: every function is pinned by a test in ``tests/`` against
values the paper prints, closed forms, library routines (np.kron,
scipy.linalg.hadamard, np.fft) or brute force; none is "parity unpinned".
"""
