"""Writes paper_pair_readings.json: the oracle's final term count, ground
energy and the exact coefficients of the energy's Pauli terms (hex floats)
for the N = 12 open chain of Sec. III.C (J = 1, h = 0.5, dtau = 0.04,
tau = 20, 500 layers from the identity) at delta = 2^-7 and 2^-8, under the
readings the oracle takes (theta = alpha dtau, threshold on the merged
coefficients before the normalisation to c_I = 1).  The paper prints, for
delta = 2^-7, about 42,466 terms and a relative ground-energy error near
1e-2; the stored values record what this reading gives instead.  Calls
only the oracle and the exact free-fermion energy; takes about two minutes.

    python tests/golden/make_paper_pair.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle                      # noqa: E402
import workloads as wl             # noqa: E402
from oracle import dense           # noqa: E402

N, J, h, dtau, tau = 12, 1.0, 0.5, 0.04, 20.0


def main():
    L = int(round(tau / dtau))
    H = wl.tfim_1d(N, J, h)
    E0 = dense.bdg_ground_energy(J, [h] * N)
    obs = wl.energy_observable(H)
    out = {"_comment": ("oracle values for the printed pair of Sec. III.C (delta = 2^-7: about "
                        "42,466 terms, relative error about 1e-2), written by "
                        "make_paper_pair.py; reading R1 does not reproduce the pair"),
           "workload": "1D open TFIM, N=12, J=1, h=0.5, dtau=0.04, 500 layers from the identity",
           "E0_free_fermion": E0, "cases": []}
    for e in (7, 8):
        o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, 2.0 ** -e)
        mx = 1
        for _ in range(L):
            o.apply_layers(1)
            mx = max(mx, o.count())
        E = o.expect(obs)
        cs = o.coeffs(obs.x, obs.z)
        out["cases"].append({"delta_log2": -e, "final_terms": o.count(), "max_terms": mx,
                             "energy": E, "rel_err": abs(E - E0) / abs(E0),
                             "energy_term_coeffs_hex": [float(c).hex() for c in cs]})
        o.close()
    with open(os.path.join(HERE, "paper_pair_readings.json"), "w") as f:
        json.dump(out, f, indent=2)


if __name__ == "__main__":
    main()
