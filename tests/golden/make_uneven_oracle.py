"""Writes uneven_5_25keV_450um_oracle200.json: the FP64 oracle's results for the
first 200 events of the uneven 5-25 keV / 450 um workload.

    python tests/golden/make_uneven_oracle.py [--events 200] [--batch 16]

Imports only ``oracle`` (the FP64 CPU implementation) and ``workloads`` (the
seeded inputs).  Every event is the preset's own descriptor (master seed
20250611, event ids 0..199, energies uniform on 5-25 keV, depths from the
workload's attenuation law).  Results are appended batch by batch to a
``.partial`` file next to the output, so an interrupted run resumes where it
stopped; the final file holds, per event, the carrier count, the oracle's step
count, its collected / outside counts and the 9 x 9 pixel map.  The cluster
size and the 3 x 3 single-pixel spectrum (Sec. 4.2) follow from the map.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

NAME = "uneven_5_25keV_450um"
OUT = os.path.join(HERE, f"{NAME}_oracle200.json")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=200)
    ap.add_argument("--batch", type=int, default=16)
    args = ap.parse_args()
    oracle.build()
    p = W.preset(NAME)
    params = oracle.make_params(p["sensor"], W.field_switches(), p["mobility"])
    evs = W.make_events(NAME, n=args.events)
    partial = OUT + ".partial"
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                rec = json.loads(line)
                done[rec["event_id"]] = rec
    todo = [e for e in evs if e["event_id"] not in done]
    t0 = time.time()
    for b in range(0, len(todo), args.batch):
        chunk = todo[b:b + args.batch]
        res = oracle.run_events(params, chunk)
        with open(partial, "a") as f:
            for e, r in zip(chunk, res):
                rec = dict(event_id=int(e["event_id"]), energy_keV=float(e["energy_keV"]),
                           depth_um=float(e["depth_um"]), n_carriers=int(len(r.state)),
                           status=int(r.status), n_steps=int(r.n_steps),
                           n_collected=int(r.n_collected), n_outside=int(r.n_outside),
                           interactions=int(r.interactions),
                           pixels=r.pixels.astype(int).tolist())
                f.write(json.dumps(rec) + "\n")
                done[rec["event_id"]] = rec
        print(f"{len(done)}/{len(evs)} events, {time.time() - t0:.0f} s", flush=True)
    with open(oracle._SRC, "rb") as f:
        src_hash = hashlib.sha256(f.read()).hexdigest()[:16]
    out = dict(
        workload=NAME, master_seed=W.MASTER_SEED, events=len(evs),
        command="python tests/golden/make_uneven_oracle.py --events %d" % len(evs),
        oracle_source_sha256_16=src_hash, oracle_threads=oracle.max_threads(),
        results=[done[e["event_id"]] for e in evs])
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    os.remove(partial)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
