"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

Usage: python tests/golden/make_golden.py [name ...]
Each file records, per coarse-graining step of the 4D Ising model, the values the
CUDA path is compared with: ln Z/V of the 2^k-site lattice, ln c_k, the discarded
eigenvalue sums of both HOSVD sides, the side taken, the new bond dimensions and
whether the cut fell inside an eigenvalue cluster. Impure runs add <sigma>,
<sigma sigma> and E/V.
"""

import json
import math
import os
import sys
import time

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))

from oracle import hotrg as H  # noqa: E402

RUNS = {
    # 4D Ising, T = 6.65, h = 0, D_cut = 4, 16 steps (16^4 lattice)
    "ising4d_T6.65_h0_dcut4_16steps": dict(T=6.65, h=0.0, dcut=4, steps=16, impure=False),
    # same with the impure tensors and a small field
    "ising4d_T6.65_h1e-5_dcut4_impure_12steps": dict(T=6.65, h=1e-5, dcut=4, steps=12, impure=True),
    # odd cut, five steps
    "ising4d_T6.65_h0_dcut5_8steps": dict(T=6.65, h=0.0, dcut=5, steps=8, impure=False),
    # 4D Ising, T = 6.65, h = 0, D_cut = 8: the first 8 of the 40 steps to 1024^4
    "ising4d_T6.65_h0_dcut8_8steps": dict(T=6.65, h=0.0, dcut=8, steps=8, impure=False),
}


def make(name):
    cfg = RUNS[name]
    st = H.HOTRG.start(4, 1.0 / cfg["T"], cfg["h"], cfg["impure"])
    steps = []
    t0 = time.time()
    for i in range(cfg["steps"]):
        r = st.step(i % 4, cfg["dcut"])
        rec = dict(k=i + 1, mu=r.mu, dims=list(r.dims_out), lnZ=r.lnZ, ln_c=r.ln_c,
                   eps={str(n): list(v) for n, v in r.eps.items()},
                   primed={str(n): bool(v) for n, v in r.primed.items()},
                   degenerate_cut=bool(r.degenerate_cut))
        if cfg["impure"]:
            rec.update(m=st.magnetization(), sigma_sigma=st.sigma_sigma(), energy=st.energy())
        steps.append(rec)
        print(name, i + 1, f"{time.time() - t0:.1f}s", r.lnZ, flush=True)
    out = dict(name=name, source="oracle/hotrg.py (FP64 NumPy), tests/golden/make_golden.py",
               d=4, beta=1.0 / cfg["T"], config=cfg, lnz_acc=st.lnz_acc, steps=steps)
    with open(os.path.join(os.path.dirname(__file__), name + ".json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(RUNS)):
        make(n)
