"""Plain FP64 CPU oracle for the coupled lattice-Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code, tables or constants with the
CUDA path under ``paper_1406_2211_gb300/``; the only module both sides use is
``synth`` (seeded input generators, no method arithmetic).

Source: U. D. Schiller, "A unified operator splitting approach for
multi-scale fluid-particle coupling in the lattice Boltzmann method"
(arXiv:1406.2211).  Each function cites the section / equation it follows.
Equation references use the paper's LaTeX labels, e.g. Eq. [csc] is the
collide-stream-collide system of Sec. 4.

Modules
  lattice   D3Q19 velocity set, equilibrium, Hermite force term, MRT basis
  lb        streaming, collision, force operators; literal CSC step (O1) and
            the exactly recombined step (O2)
  delta     discrete delta functions (App. A) and interpolation / spreading
            (Sec. 5.1)
  coupling  IBM / force coupling / EBF / modified EBF operators (Sec. 5),
            first- and second-order schemes, multiple time steps (Sec. 6)
  sim       a simulation box that strings the operators into time steps
  fluct     fluctuating MRT collision (Eq. [mrt-fluct]) with a counter-based
            random number generator; recombined and literal fluctuating steps

Parity pins (what ties each part to the paper rather than to itself) are
the tests in tests/test_oracle_*.py.  Parts without an independent pin are
listed in the module headers as "parity unpinned".
"""
