"""Writes the oracle's ln Z values that the GPU evidence tests compare against.

Calls only the oracle (and the seeded input recipes): each workload's event is
the oracle waveform at the injection plus seeded noise (tests/helpers.py), and
each ln Z is one full oracle SMC-NUTS run (Sec. 3: adaptive tempering,
systematic resampling, NUTS mutations; Sec. 3.1, Eqs. 7-8: the evidence as the
sum of the stage increments) with its own key. Nothing here touches the CUDA
library.

    python tests/golden/make_lnz_oracle.py bbh11 [R [DIR]]   # 2048 particles, depth 6, identity metric
    python tests/golden/make_lnz_oracle.py batch1 [R [DIR]]  # one event of the batched recipe, 256 particles

Writes DIR/lnz_<name>_oracle.json (DIR defaults to tests/golden).
"""
import json
import os
import platform
import sys
import time

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

import oracle  # noqa: E402
from paper_2601_02336_gb300 import inputs  # noqa: E402
from tests import helpers  # noqa: E402


def workload(name):
    if name == "bbh11":
        return inputs.bbh11(), 0, 5000
    if name == "batch1":
        # event 5 of the batched recipe (a 4 s segment) with 256 particles, depth 8
        w = inputs.batch64()[5]
        w.n_particles = 256
        return w, 5, 6000
    raise SystemExit(f"unknown workload {name}")


def main():
    name = sys.argv[1]
    reps = int(sys.argv[2]) if len(sys.argv) > 2 else 10
    out_dir = sys.argv[3] if len(sys.argv) > 3 else os.path.dirname(os.path.abspath(__file__))
    w, seed, key0 = workload(name)
    ev, th_inj, _ = helpers.make_event(w, seed)
    model = helpers.oracle_model(w)
    oracle.set_threads(os.cpu_count() or 1)
    runs = []
    for r in range(reps):
        t0 = time.time()
        lnz, _, _, rec = oracle.smc_run(model, ev, w.n_particles, w.alpha, w.n_mut, w.max_depth, w.metric,
                                        w.eps_scale, key=key0 + r)
        runs.append({"key": key0 + r, "lnz": lnz, "stages": len(rec),
                     "evals": int(sum(s["n_leapfrog"] for s in rec))})
        print(f"run {r}: key {key0 + r} ln Z {lnz:.6f} stages {len(rec)} ({time.time() - t0:.0f} s)", flush=True)
    out = {
        "script": "tests/golden/make_lnz_oracle.py",
        "what": "ln Z of full oracle SMC-NUTS runs (Sec. 3, Sec. 3.1 Eqs. 7-8), one per key",
        "workload": w.name, "event_seed": seed, "n_particles": w.n_particles, "n_bins": w.n_bins,
        "df": w.df, "max_depth": w.max_depth, "alpha": w.alpha, "n_mut": w.n_mut, "metric": w.metric,
        "eps_scale": w.eps_scale, "host": f"{platform.machine()}, {os.cpu_count()} threads", "runs": runs,
    }
    path = os.path.join(out_dir, f"lnz_{name}_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
