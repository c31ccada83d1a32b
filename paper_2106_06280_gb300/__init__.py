"""GB300-native RKDG + compact-subcell-WENO (CSWENO) solver on unstructured
triangles (arXiv 2106.06280).  The CUDA library is loaded on first use by
``paper_2106_06280_gb300.cswdg``; ``workloads`` is pure numpy."""
