"""Autotune the launch shapes of the sum-factorisation kernels (elements and
threads per CTA of the volume and lift kernels) for each (dim, P, Q) of the
workloads and write the tuning table tuning.json beside this file.

    python -m paper_2002_04222_gb300.tune          # on a GPU
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def cases():
    import workloads as w
    yield w.vortex_case(n=8, P=2)
    for P in range(1, 7):
        yield w.poiseuille_case(P)
    yield w.tgv_case(n=16, P=3)
    yield w.tgv_case(n=16, P=4, Q=8)
    yield w.tgv_case(n=16, P=2, Q=5)


def main(reps=10):
    import paper_2002_04222_gb300 as dgl
    table = {}
    for c in cases():
        m = dgl.Mesh.from_case(c)
        key = f"{m.info['dim']}d_P{m.info['P']}_Q{m.info['Q']}"
        r = dgl.autotune(m, reps=reps)
        r["workload"] = c.name
        table[key] = r
        print(key, r, flush=True)
        m.close()
    with open(dgl.TUNING_TABLE, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print("wrote", dgl.TUNING_TABLE)


if __name__ == "__main__":
    main()
