"""Writes tissue_serial_stats_128.json: the statistics of tests/tissue_stats.py
for the serial CPM chain (oracle (a): Methods, Eq. 1-3, Eq. 8-9, one
uniformly drawn attempt at a time) on the 128^3 Act fibre tissue, one entry
per seed.  Calls only the oracle and the seeded input generators; the GPU
test compares the parallel scheme's 64-seed means with these.

    python tests/golden/make_tissue_serial_stats.py [n_procs]

About 8 CPU-hours (64 seeds x 500 MCS x 2.1 M attempts, bound by the
lattice's cache misses); finished seeds are kept under _build/ and reused
when the script is run again."""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

SEEDS = list(range(1, 65))
OUT = os.path.join(HERE, "tissue_serial_stats_128.json")
PARTS = os.path.join(ROOT, "_build", "tissue_serial_parts")  # one finished seed per file (resumable)


def run(seed):
    part = os.path.join(PARTS, "seed_%03d.json" % seed)
    if os.path.exists(part):
        return seed, json.load(open(part))
    import cpm_workloads as cw
    import oracle
    import tissue_stats as ts
    # the workload's fibre mask is drawn with torch on the CPU: one thread per process
    import torch
    torch.set_num_threads(1)
    w = cw.fibre_tissue_3d(seed=seed, n=ts.N)
    st = oracle.State(w)
    st.serial_run(ts.BURN)
    rec = ts.Recorder((w.nz, w.ny, w.nx), w.n_cells)
    shape = (w.nz, w.ny, w.nx)
    rec.snapshot(st.lattice.reshape(shape))
    acc = 0
    for _ in range(ts.SNAPS):
        acc += st.serial_run(ts.EVERY)
        rec.snapshot(st.lattice.reshape(shape), st.V, st.A)
    out = rec.summary(acc, w.n_sites)
    tmp = part + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(out, f)
    os.replace(tmp, part)
    return seed, out


def main():
    n_procs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    os.makedirs(PARTS, exist_ok=True)
    t0 = time.time()
    with mp.get_context("spawn").Pool(n_procs, maxtasksperchild=1) as pool:
        res = dict(pool.imap_unordered(run, SEEDS))
    import tissue_stats as ts
    doc = {
        "what": "serial CPM chain (oracle (a)) statistics of the 128^3 Act fibre tissue, per seed",
        "protocol": {"n": ts.N, "burn_mcs": ts.BURN, "snapshots": ts.SNAPS, "every_mcs": ts.EVERY},
        "seeds": SEEDS,
        "stats": {k: [res[s][k] for s in SEEDS] for k in ts.STATS},
        "cpu_seconds": round((time.time() - t0) * n_procs),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT, "in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
