"""Writes mcrit.json: the critical mass m_c of each synthetic gauge field used by the
workloads, computed by the FP64 oracle (oracle.spectrum: m_c = -min Re lambda(D(0))).

Run from the repository root:  python tests/golden/make_mcrit.py [--only L,beta]
Each entry records the generator recipe, the digest of the link angles (identical on
every host: the chain depends on libm only through accept decisions) and m_c.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
from oracle import spectrum  # noqa: E402
from oracle.lattice import Lattice  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mcrit.json")

# (workload id, L, beta): 64^2 beta=6 (the small two-level case), the 256^2 points
# of the three-level sweep over beta in {3, 6, 10}, and a 128^2 beta=6 field
FIELDS = [(0, 64, 6.0), (1, 256, 3.0), (1, 256, 6.0), (1, 256, 10.0),
          (2, 128, 6.0)]  # the mixed-size batch (64^2, 128^2 and 256^2 fields)
# (workload id, L, beta) of fields too large for the Arnoldi scan (the 1024^2 points of the
# three-level sweep): m_c is taken from the 256^2 field of the same beta and recipe (a calibration
# on the smaller lattice), and the row records the 1024^2 field's own digest
CALIBRATED = [(1, 1024, 3.0), (1, 1024, 6.0), (1, 1024, 10.0)]
CALIBRATION_L = 256
# (workload id, dims) of the 4d SU(3) fields: projected 1 + 0.4 H links after 4 APE steps (alpha 0.5)
FIELDS4 = [(3, (16, 16, 16, 32))]
# a smaller lattice of the same 4d recipe: when the Arnoldi scan of the 16^3 x 32 field is too slow,
# its m_c is taken from this calibration (as the 1024^2 fields take theirs from 256^2)
CALIBRATION4 = (8, 8, 8, 16)


def key4(wid, dims):
    return f"w{wid}_su3_" + "x".join(str(d) for d in dims)


def key(wid, L, beta):
    return f"w{wid}_L{L}_b{beta:g}"


def save(k, row):
    """Merge one entry into the stored table (re-read first: several scans may run at once)."""
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    table[k] = row
    json.dump(table, open(OUT, "w"), indent=1, sort_keys=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    ap.add_argument("--su3", action="store_true", help="the 4d SU(3) fields only")
    ap.add_argument("--calibrated", action="store_true", help="the 1024^2 fields (m_c from 256^2)")
    ap.add_argument("--su3-calibrated", action="store_true",
                    help="the 4d fields with m_c from the 8^3 x 16 field of the same recipe")
    args = ap.parse_args()
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if args.calibrated:
        for wid, L, beta in CALIBRATED:
            if args.only and args.only != f"{L},{beta:g}":
                continue
            src = key(wid, CALIBRATION_L, beta)
            if src not in table:
                raise SystemExit(f"{src} must be computed first")
            t0 = time.time()
            U, theta, acc = inputs.schwinger_links(L, beta, sweeps=2000, workload_id=wid)
            t1 = time.time()
            row = dict(workload_id=wid, L=L, beta=beta, sweeps=2000, hits=10, step=0.5,
                       seed=inputs.workload_seed(wid, L, beta), acceptance=acc,
                       Q=round(inputs.topological_charge(theta, L, L)), theta_digest=inputs.field_digest(theta),
                       m_crit=table[src]["m_crit"], m_crit_from=src, gen_seconds=round(t1 - t0, 1))
            print(key(wid, L, beta), row, flush=True)
            save(key(wid, L, beta), row)
        return
    if args.su3_calibrated:
        for wid, dims in FIELDS4:
            t0 = time.time()
            Uc = inputs.su3_links(CALIBRATION4, seed=inputs.workload_seed(wid, CALIBRATION4[0], 0.0))
            mc = spectrum.critical_mass_arnoldi(Uc, Lattice(CALIBRATION4), Nc=3, k=4, ncv=40, tol=1e-6)
            t1 = time.time()
            src = key4(wid, CALIBRATION4)
            save(src, dict(workload_id=wid, dims=list(CALIBRATION4), eps=0.4, ape_steps=4, ape_alpha=0.5,
                           seed=inputs.workload_seed(wid, CALIBRATION4[0], 0.0),
                           links_digest=inputs.field_digest(Uc), m_crit=mc, scan_seconds=round(t1 - t0, 1)))
            U = inputs.su3_links(dims, seed=inputs.workload_seed(wid, dims[0], 0.0))
            row = dict(workload_id=wid, dims=list(dims), eps=0.4, ape_steps=4, ape_alpha=0.5,
                       seed=inputs.workload_seed(wid, dims[0], 0.0), links_digest=inputs.field_digest(U),
                       m_crit=mc, m_crit_from=src)
            print(src, mc, key4(wid, dims), row, flush=True)
            save(key4(wid, dims), row)
        return
    if args.su3:
        for wid, dims in FIELDS4:
            t0 = time.time()
            U = inputs.su3_links(dims, seed=inputs.workload_seed(wid, dims[0], 0.0))
            t1 = time.time()
            # m_c to about 1e-4 is enough to place m = m_c + 0.005: a looser Arnoldi tolerance
            mc = spectrum.critical_mass_arnoldi(U, Lattice(dims), Nc=3, k=4, ncv=40, tol=1e-4)
            t2 = time.time()
            table[key4(wid, dims)] = dict(workload_id=wid, dims=list(dims), eps=0.4, ape_steps=4, ape_alpha=0.5,
                                          seed=inputs.workload_seed(wid, dims[0], 0.0),
                                          links_digest=inputs.field_digest(U), m_crit=mc,
                                          gen_seconds=round(t1 - t0, 1), scan_seconds=round(t2 - t1, 1))
            print(key4(wid, dims), table[key4(wid, dims)], flush=True)
            save(key4(wid, dims), table[key4(wid, dims)])
        return
    for wid, L, beta in FIELDS:
        if args.only and args.only != f"{L},{beta:g}":
            continue
        t0 = time.time()
        U, theta, acc = inputs.schwinger_links(L, beta, sweeps=2000, workload_id=wid)
        t1 = time.time()
        lat = Lattice((L, L))
        mc = spectrum.critical_mass(U, lat)
        t2 = time.time()
        table[key(wid, L, beta)] = dict(workload_id=wid, L=L, beta=beta, sweeps=2000, hits=10, step=0.5,
                                        seed=inputs.workload_seed(wid, L, beta), acceptance=acc,
                                        Q=round(inputs.topological_charge(theta, L, L)),
                                        theta_digest=inputs.field_digest(theta), m_crit=mc,
                                        gen_seconds=round(t1 - t0, 1), scan_seconds=round(t2 - t1, 1))
        print(key(wid, L, beta), table[key(wid, L, beta)], flush=True)
        save(key(wid, L, beta), table[key(wid, L, beta)])


if __name__ == "__main__":
    main()
