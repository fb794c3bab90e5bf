"""FP64 CPU oracle for the HOTRG coarse-graining step of the Ising model.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain reference that the CUDA
path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never does.

Modules
-------
hotrg  : the HOTRG algorithm in FP64 NumPy, any dimension d (Sec. 2, Fig. 1 of
         arXiv:1911.12954, with the site tensor and impure-tensor scheme).
atrg   : the anisotropic TRG (Sec. 2, Fig. 2; Sec. 3.2) in FP64 NumPy, any d: the SVD of
         each local tensor, the index swap by a truncated (or randomized) SVD, the HOSVD
         of the two decomposed halves, the contraction.
exact  : independent closed forms and brute force used to pin ``hotrg`` and ``atrg``: exact
         enumeration of small periodic lattices, Onsager's 2D free energy, the 2D
         internal energy and Yang's magnetisation, and the hypercubic
         high-temperature series.

Parity status: every function in ``hotrg`` is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` (enumeration, Onsager, series, brute-force
contraction, symmetry), every function in ``atrg`` in ``tests/test_atrg_pins.py``
(enumeration without truncation, Onsager with it, the exact SVD for the randomized
one). Nothing here is "parity unpinned".
"""
