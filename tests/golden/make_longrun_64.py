"""Write ``longrun_64_oracle.txt``: time averages of a long forced run of the
FP64 oracle, the expected values of ``tests/test_gpu_longrun.py``.

The run (section 2.3 workflow; Table 1 and Fig. 2b records): 64^3, random-phase
solenoidal IC with E(k) ~ k^4 exp(-2 (k/4)^2) and K = 1.5 (seed 2), nu from
k_max eta = 1.5 (k_max = N/3, eps = 0.1), Sc = 1, beta = 1, constant-power
forcing eps_inj = 0.1 on 0 < |k| <= 2, CFL 0.5 (Eq. 10; dt reset at every
record), Lawson IF-RK4, 2000 steps, a record every 10 steps (201 records).
Stored: means over all records and over the second half of the records (the
101 records from step 1000 on) of E(n) for every shell and of eps, eps_phys,
chi and K, and the final time.  Calls the oracle only.

    python tests/golden/make_longrun_64.py      # about 15 minutes on one core
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import psc_oracle as O  # noqa: E402

N, STEPS, EVERY, SEED = 64, 2000, 10, 2


def params():
    eta = 1.5 / (N / 3.0)
    nu = (eta ** 4 * 0.1) ** (1.0 / 3.0)
    return O.Params(N=N, nu=nu, Sc=1.0, beta=1.0, forcing=O.FORCE_CONST_POWER, kF=2.0, eps_inj=0.1,
                    cfl=0.5, dt=0.01, seed=SEED, ic=O.IC_SPECTRUM_K4, ic_energy=1.5, record_every=EVERY)


def main():
    p = params()
    _, _, recs, t, _ = O.run(p, STEPS)
    keys = ("eps", "eps_phys", "chi", "K")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "longrun_64_oracle.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, written by tests/golden/make_longrun_64.py (see its docstring)\n")
        f.write(f"# N={N} nu={p.nu!r} steps={STEPS} record_every={EVERY} records={len(recs)} seed={SEED}\n")
        f.write(f"t_final {t!r}\n")
        for tag, rs in (("all", recs), ("half", recs[len(recs) // 2:])):
            for k in keys:
                f.write(f"{tag} {k} {float(np.mean([r[k] for r in rs]))!r}\n")
            E = np.mean([r["E"] for r in rs], axis=0)
            for n, e in enumerate(E):
                f.write(f"{tag} E{n} {float(e)!r}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
