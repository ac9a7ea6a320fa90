"""CPU oracle for the PDX search path.

TEST INFRASTRUCTURE ONLY: this package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``, and by
nothing else. It never imports the CUDA package and the CUDA package never
imports it. It is plain and slow on purpose: FP64 arithmetic on the float32
inputs, whole-array sorts, no blocking or fusion.

Modules:
  knn        ctypes wrapper over ``knn_oracle.c`` (brute-force top-k, probed
             buckets, nearest centroid, Lloyd k-means) -- plain definitions.
  pdxearch   the PDXearch framework (Sec. 4) with the PDX-BOND (Sec. 5),
             ADSampling and BSA pruning predicates, block by block in the
             paper's order.
  quant      element-wise quantisation to BF16 / FP8-E4M3 and the error bound
             that the low-precision scan widens its prune test by.
  mlp        FP64 forward/backward of the 2-layer order-proposal network.
"""
from . import knn  # noqa: F401
