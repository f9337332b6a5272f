"""Plain FP64 CPU oracle for the hierarchical-H-matrix PCG method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline and ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA path;
both sides read their inputs from the ``inputs`` generator module.

Each function follows the paper's definition in its own plain form (loops,
numpy, LAPACK through scipy, plain PyTorch CPU ops in float64 for the network)
and cites the passage it implements.  Modules:

* ``rng``      counter-based SplitMix64 (Steele, Lea & Flood 2014)
* ``grid``     Morton ordering and operator assembly (Supp. D, Sec. 7.1)
* ``hmatrix``  weak-admissibility partition, packed factor layouts, SVD-H
               construction, dense M, structured apply (Sec. 4, Sec. 5, Supp. B)
* ``pcg``      preconditioned CG with FP64 scalars (Sec. 5, Sec. 6.3, Supp. G)
* ``loss``     cosine-Hutchinson loss and probes (Sec. 6.1, Eq. 7, Eq. 8)
* ``network``  the hierarchical transformer forward pass (Sec. 4, Supp. B)
* ``adamw``    AdamW with global-norm clipping (Supp. C)
* ``train``    batch loss and its gradient by autograd through ``network`` (Sec. 6, Supp. C)
* ``diagnostics`` spectrum of M A and the off-diagonal rank audit (Fig. 1, Fig. 3)

Pins for every function live in ``tests/test_oracle_*.py``.
"""
