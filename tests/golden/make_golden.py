"""Writes the oracle-computed fixtures of this folder.  It calls only the
oracle (and the seeded input generators), so every stored value comes from
the plain binary64 restatement of the method, never from the CUDA path.

    python tests/golden/make_golden.py

Fixture: pod_waves_2048x24.txt -- the POD (Alg. 2 through Eqs. svdqr1-3 of
Sec. 3.1: mean removal, sqrt(cell-volume) weights, QR, SVD of R, energy
truncation of Sec. 3.1) of a seeded 2048 x 24 traveling-wave field with
log-uniform cell volumes, at 99 % energy."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the case: shared with the tests that read the fixture
POD_CASE = dict(N=2048, M=24, n_waves=6, noise=1e-3, seed=11, w_seed=12, energy=0.99)
POD_FILE = os.path.join(HERE, "pod_waves_2048x24.txt")
MEAN_ROWS = (0, 1, 511, 1024, 2047)


def pod_case_inputs():
    import synth
    c = POD_CASE
    X = synth.waves(c["N"], c["M"], n_waves=c["n_waves"], noise=c["noise"], seed=c["seed"])
    w = synth.log_uniform_weights(c["N"], seed=c["w_seed"])
    return X, w


def write_pod():
    import oracle
    X, w = pod_case_inputs()
    res = oracle.pod(X, w=w, remove_mean=True, energy=POD_CASE["energy"])
    lines = [
        "# POD of a seeded 2048 x 24 traveling-wave field (synth.waves: 6 waves, noise 1e-3, seed 11),",
        "# cell volumes synth.log_uniform_weights(seed 12), temporal mean removed, 99 % energy.",
        "# Alg. 2 via Eqs. svdqr1-3 (Sec. 3.1); truncation by the accumulated energy (Sec. 3.1).",
        "# Written by tests/golden/make_golden.py from oracle.pod (binary64).",
        f"r {res['r']}",
    ]
    lines += [f"S {i} {s:.17e}" for i, s in enumerate(res["S"])]
    lines += [f"mean {n} {res['mean'][n]:.17e}" for n in MEAN_ROWS]
    with open(POD_FILE, "w") as f:
        f.write("\n".join(lines) + "\n")


def read_fixture(path):
    """{key: value or [(index, value), ...]} of a fixture file."""
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if len(parts) == 2:
            out[parts[0]] = float(parts[1])
        else:
            out.setdefault(parts[0], []).append((int(parts[1]), float(parts[2])))
    return out


if __name__ == "__main__":
    write_pod()
    print("wrote", POD_FILE)
