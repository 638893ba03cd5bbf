"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

This package is the independent, slow, obviously correct statement of what
the GPU path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_2507_15277_gb300/`` never does, and the two share no code (only the
seeded input generators in ``workloads/``).

Modules:
  gemm    FP64-accumulating GEMM (C source ``gemm_ref.c``), the definition of
          the operation.
  select  Portability tuning arithmetic: per-shape best ("Oracle" in the
          paper's sense), the set cost function (Eq. 1), exhaustive
          PortabilityTune over k-subsets, post-processing (Table 5),
          search-space size, the k-means and decision-tree selections, and
          the shape -> variant rule of the runtime selector.
  checks  The normalised error used by every parity test.
"""
