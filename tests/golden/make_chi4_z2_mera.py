"""Writes tests/golden/mera_chi4_z2.json: a chi = 4 scale-invariant binary
MERA for the critical Ising chain optimised by the FP64 oracle alone.

Start: init_mera(seed=0, chi=4, z2=True) (parity-symmetric isometric
tensors), rho* = 1/chi^3.  Then SWEEPS oracle sweeps (Sec. II C, 20 power
steps of rho* each).  The file holds every layer's u and w, rho*, and the
oracle's energy per spin of the final state.  Only oracle/ and the seeded
input generators are called.

    python tests/golden/make_chi4_z2_mera.py      # about 10 minutes on 8 cores
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import mera_inputs as I  # noqa: E402
from oracle import mera_oracle as O  # noqa: E402

SEED, CHI, SWEEPS, N_POW = 0, 4, 8900, 20
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mera_chi4_z2.json")


def main():
    layers = I.init_mera(SEED, CHI, z2=True)
    h1, shift = O.ising_h1(1.0)
    rho = O.identity_density(CHI)
    for _ in range(SWEEPS):
        layers, rho, _ = O.sweep(layers, h1, shift, rho, N_POW)
    e = O.energy_per_spin(layers, h1, shift, rho, 100)
    doc = {
        "_source": "written by tests/golden/make_chi4_z2_mera.py from the FP64 oracle only",
        "seed": SEED, "chi": CHI, "sweeps": SWEEPS, "n_pow": N_POW, "hz": 1.0, "z2": True,
        "energy_per_spin": e,
        "layers": [{"u": u.reshape(-1).tolist(), "w": w.reshape(-1).tolist(),
                    "chi_b": int(w.shape[0]), "chi_t": int(w.shape[2])} for u, w in layers],
        "rho_star": rho.reshape(-1).tolist(),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, separators=(",", ":"))
        f.write("\n")
    print(f"{OUT}: energy per spin {e:.12f} (exact {O.exact_energy_per_spin(1.0):.12f})")


if __name__ == "__main__":
    main()
