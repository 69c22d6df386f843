"""FP64 CPU oracle for unbalanced entropic domain decomposition.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the paper's mathematics (Medina, Nguyen,
Schmitzer, "Domain decomposition for entropic unbalanced optimal transport")
in NumPy float64.  It exists to check the CUDA path.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it; the product library never does, and it shares no
code with the CUDA path.

Modules
  uot     -- divergences, primal/dual scores, global Sinkhorn (Sections 2.2, 5.1)
  cell    -- cell subproblem: Y-half root, cell Sinkhorn, PD stopping (Section 5.1)
  domdec  -- partitions, parallel / sequential DomDec, GetWeights, bookkeeping
             (Sections 2.3, 3.1, 4.3, 5.1-5.3)
  brute   -- damped Newton maximisation of the dual on tiny problems (pins)

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, brute-force convex
maximisation, identities, invariants), except where a docstring says
"parity unpinned".
"""
