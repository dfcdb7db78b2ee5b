"""Oracle: plain, slow, obviously correct CPU (numpy, fp64) restatement of the
SFFT-based homogenisation method, used ONLY as test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA
library never calls it, and it shares no code with the CUDA library: the only
module both sides use is the seeded geometry generator
``paper_2412_11566_gb300.synth``, which holds none of the method's arithmetic.

Modules:
  dense  -- Oracle A: the dense FFT basic scheme (Alg. 1) and C_eff by unit loads,
            with the six discretisation schemes of App. A's table.
  dense2d -- Oracle A in 2D (plane strain, 3-component Voigt form), written
            without dense's Green operator so that the two can be compared.
  qtt    -- Oracle B: tensor-train primitives, the SFFT/Green/stiffness operators
            and the SFFT-based scheme (Alg. 2), in the same step order as the
            CUDA path so that FP64 results can be compared to 1e-10; also the
            paper's own constructions the CUDA path replaces, to compare with:
            the SFFT MPO from the QFT circuit by zip-up (Sec. 4.2), the
            AMEn-adapted product (App. B), the randomized TT-SVD (App. D),
            and the 2D controlled QTT with a 3-component Voigt core.

Every function names the passage of the paper it restates.

Pins (tests/test_oracle_*.py, no GPU): the Green operator against its
definition and projector identities, and every difference scheme (3D and 2D)
against a brute-force real-space operator D (D^T C0 D)^+ D^T; 2D against the
3D oracle on the extruded section; the FFT against a
brute-force DFT; homogeneous medium, laminate closed form, the LU solution of
the discrete LS system, Voigt/Reuss/Hashin-Shtrikman bounds; broadcast grids
against full grids; SFFT MPO rank and unitarity; rounding error bound; exact
product rank; the sketched product exact at its true rank and quasi-optimal
on flat spectra, with planted mistakes that fail; Philox known answers; the
two oracles against each other; and, between those two cases, the sketched
product on the Green product of an LS iteration truncated to ranks 8-24,
within 10 % of the TT-SVD of the dense product for every seed tried (and the
AMEn product of App. B with it).
"""
