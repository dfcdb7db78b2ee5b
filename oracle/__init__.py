"""Oracle: plain, slow, obviously correct CPU (numpy, fp64) restatement of the
SFFT-based homogenisation method, used ONLY as test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA
library never calls it, and it shares no code with the CUDA library: the only
module both sides use is the seeded geometry generator
``paper_2412_11566_gb300.synth``, which holds none of the method's arithmetic.

Modules:
  dense  -- Oracle A: the dense FFT basic scheme (Alg. 1) and C_eff by unit loads.
  qtt    -- Oracle B: tensor-train primitives, the SFFT/Green/stiffness operators
            and the SFFT-based scheme (Alg. 2), in the same step order as the
            CUDA path so that FP64 results can be compared to 1e-10.

Every function names the passage of the paper it restates.

Pins (tests/test_oracle_*.py, no GPU): the Green operator (Direct and
Centered) against its definition and projector identities; the FFT against a
brute-force DFT; homogeneous medium, laminate closed form, the LU solution of
the discrete LS system, Voigt/Reuss/Hashin-Shtrikman bounds; broadcast grids
against full grids; SFFT MPO rank and unitarity; rounding error bound; exact
product rank; the sketched product exact at its true rank and quasi-optimal
on flat spectra, with planted mistakes that fail; Philox known answers; the
two oracles against each other. Between its exact and its flat-spectrum case
the sketched product's error is measured, not bounded (parity unpinned there).
"""
