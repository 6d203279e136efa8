"""Write tests/golden/oracle_8x8_seed1.json from the CPU oracle alone.

The stored values are the oracle's own outputs on the 8^4, beta = 1, seed 1
workload (20 compound sweeps of 1 Metropolis + 3 overrelaxation passes, then
one multilevel level with slabs of 2 slices).  They are bit-exact doubles
(hex) and pin the oracle's arithmetic across machines: the x86 build host and
the aarch64 GPU host must reproduce them exactly.

Run:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def compute():
    lat = O.Lattice(8, 8, 1.0, 1)
    for _ in range(20):
        lat.sweep(1, 3)
    out = {
        "workload": "8^4 beta=1.0 seed=1, 20 sweeps (1 Metropolis width 1.0 + 3 OR), "
                    "then multilevel slab_t=2 n_sub=6 (1+3 passes) r<=3 d<=2",
        "plaquette_after_20": lat.plaquette().hex(),
        "theta_sample_after_20": [float(lat.theta[k]).hex() for k in (0, 1, 777, 4095, 9000, 16383)],
        "metro_pass_after_20": int(lat.metro_pass.value),
    }
    ml = lat.multilevel(2, 6, 3, d_max=2, sub_metro=1, sub_or=3)
    out["corr"] = [[z.real.hex(), z.imag.hex()] for z in ml["corr"]]
    out["fields_r2_d1"] = [[z.real.hex(), z.imag.hex()] for z in ml["fields"][1, 1]]
    out["vac"] = [float(v).hex() for v in ml["vac"]]
    out["plaquette_after_level"] = lat.plaquette().hex()
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_8x8_seed1.json"), "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
