"""Write the stored expected growth vectors of the large workloads.

Every value written here comes from the CPU oracle (``oracle/``) and nothing else.  Run from
the repository root:  python tests/golden/make_golden.py [name ...]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as w  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # name: (n, gens, two_layer, max_radius, description)
    "s11_lrx_growth": (11, w.lrx(11), True, -1,
                       "S_11, LRX generators, full growth from the identity"),
    "s14_pancake_layers": (14, w.pancake(14), True, 8,
                           "S_14, 13 prefix reversals, layers 0..8 from the identity"),
    "s10_lx_growth": (10, w.lx(10), False, -1,
                                   "S_10, LX generators (directed), full growth"),
    # oracle B (visited bitmap over all n! ranks): the layers oracle A cannot hold in memory
    "s14_pancake_layers_b": (14, w.pancake(14), "bitmap", 10,
                             "S_14, 13 prefix reversals, layers 0..10 from the identity"),
    # oracle C (visited set and layers as bitmaps over all n! ranks): whole growths of S_13
    "s13_pancake_growth": (13, w.pancake(13), "bitmask", -1,
                           "S_13, 12 prefix reversals, full growth from the identity"),
    "s14_pancake_growth": (14, w.pancake(14), "bitmask", -1,
                           "S_14, 13 prefix reversals, full growth from the identity"),
    # whole S_12 growths by both large-n oracles: B (classic Lehmer rank, list frontier) and C
    # (position-major rank, layer bitmaps) share no indexing or traversal design, so equal
    # vectors pin C beyond the n <= 10 sizes where oracle A checks it
    "s12_pancake_growth_b": (12, w.pancake(12), "bitmap", -1,
                             "S_12, 11 prefix reversals, full growth from the identity"),
    "s12_pancake_growth_c": (12, w.pancake(12), "bitmask", -1,
                             "S_12, 11 prefix reversals, full growth from the identity"),
    "s12_lrx_growth_b": (12, w.lrx(12), "bitmap", -1,
                         "S_12, LRX generators, full growth from the identity"),
    "s12_lrx_growth_c": (12, w.lrx(12), "bitmask", -1,
                         "S_12, LRX generators, full growth from the identity"),
}


_BATCH = None


def _batch_one(i):
    j = _BATCH[i]
    g, rc = oracle.growth(j.n, j.gens)     # full visited set: the definition, any generator set
    assert rc == 0
    return g


def write_batch(name, workers=0):
    """Config 4: the growth vector of every one of the 4096 seeded groups (oracle A, full visited
    mode), one line per group, computed by a pool of host processes."""
    import multiprocessing as mp
    global _BATCH
    jobs = w.batch_groups()
    _BATCH = jobs
    t0 = time.time()
    ctx = mp.get_context("fork")             # no GPU in this process: fork is safe here
    with ctx.Pool(workers or os.cpu_count()) as pool:
        res = pool.map(_batch_one, range(len(jobs)), chunksize=4)
    dt = time.time() - t0
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# config 4: growth of each of the {len(jobs)} groups of workloads.batch_groups() "
                f"(seed {w.BATCH_SEED}), in index order\n")
        f.write(f"# written by tests/golden/make_golden.py from the CPU oracle (full visited mode, "
                f"{dt:.0f} s on {workers or os.cpu_count()} processes); line: index n k layer_0 layer_1 ...\n")
        for i, (j, g) in enumerate(zip(jobs, res)):
            f.write(f"{i} {j.n} {j.k} " + " ".join(str(c) for c in g) + "\n")
    print(name, len(res), sum(sum(g) for g in res), f"{dt:.1f}s")


BATCH_CASES = {"batch4096_growth": write_batch}


def write(name):
    if name in BATCH_CASES:
        return BATCH_CASES[name](name)
    n, gens, two, maxr, desc = CASES[name]
    t0 = time.time()
    if two == "bitmap":
        g, rc = oracle.growth_bitmap(n, gens, max_radius=maxr)
    elif two == "bitmask":
        g, rc = oracle.growth_bitmask(n, gens, max_radius=maxr,
                                      progress=lambda r, c: print(f"  layer {r}: {c}", flush=True))
    else:
        g, rc = oracle.growth(n, gens, two_layer=two, max_radius=maxr)
    dt = time.time() - t0
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# {desc}\n")
        mode = {"bitmap": "rank-bitmap oracle B", "bitmask": "layer-bitmap oracle C"}.get(
            two, "two-layer" if two else "full visited")
        f.write(f"# written by tests/golden/make_golden.py from the CPU oracle "
                f"({mode} mode, max_radius={maxr}, {dt:.0f} s)\n")
        for r, c in enumerate(g):
            f.write(f"{r} {c}\n")
    print(name, len(g), sum(g), f"{dt:.1f}s")


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES) + list(BATCH_CASES)):
        write(name)
