"""FP64 CPU oracle for the ArsoNISQ Monte Carlo Pauli-error path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the C-ABI library and
its Python binding) may import, call or execute this package; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.

It is a plain, slow restatement of what the paper computes, in complex128:

* ``gates``       - gate matrices from their textbook definitions
* ``statevector`` - state-vector simulation (Sec. II) and the Pauli error
                    gates of Eq. (2), appended after a gate (Sec. IV-B)
* ``philox``      - Philox4x32-10 counter RNG (Salmon et al., SC'11)
* ``sampling``    - Monte Carlo error sampling (Sec. IV-B.2)
* ``criteria``    - success criteria (Sec. II: fidelity, measurement
                    probability, binning; plus argmax)
* ``montecarlo``  - MC success probability (Sec. IV-C, last paragraph)
* ``exhaustive``  - single-error state set, Eq. (3); Eq. (4); Eq. (5)
* ``density``     - exact density-matrix Pauli channel (n <= 6), used only
                    to pin the MC estimator
* ``enumerate``   - brute-force expectation over all 4^L error patterns
* ``search``      - tolerable error rate (Sec. IV-D, Fig. 3)
* ``mlp``         - FP64 reference of the surrogate MLP's forward/backward

The oracle shares no code with the CUDA library. Its only shared input is the
seeded circuit generator in ``workloads``.
"""
