"""Small-shape sweep through the bounds-checked library (run in a child
process with EG_CHECKED_LIBRARY=1 by tests/test_gpu_checked.py): every result
must equal the oracle's and report no out-of-range index."""
import random
import sys

import numpy as np


def shapes(seed=0):
    rng = random.Random(seed)
    out = [(a,) for a in range(1, 6)]
    out += [(a, b) for a in range(1, 6) for b in range(1, 6)]
    out += [(a, b, c) for a in range(1, 6) for b in range(1, 6) for c in range(1, 6)]
    out += [tuple(rng.randint(1, 5) for _ in range(4)) for _ in range(60)]
    out += [tuple(rng.randint(1, 5) for _ in range(5)) for _ in range(40)]
    return out


def main():
    import torch

    import oracle
    from paper_2303_02724_gb300 import _build, eg, fields as F
    assert eg.LIB_PATH.endswith("libeg_checked.so"), eg.LIB_PATH
    _build.build(checked=True)
    eg.load()
    n = 0
    general = eg.EGConfig(flags=eg.EG_FLAG_NO_FUSED)
    with eg.Handle(0) as hmax, eg.Handle(0, minimum=True) as hmin, eg.Handle(0, config=general) as gmax:
        # (small 1D-3D fields take the fused kernel; gmax sends them through
        # the general launches too)
        for i, ext in enumerate(shapes()):
            for kind in ("white", "ties"):
                f = F.white_noise(ext, 100 + i) if kind == "white" else F.integer_ties(ext, 100 + i, 3)
                t = torch.from_numpy(f.values).cuda()
                for h, minimum in ((hmax, False), (hmin, True), (gmax, False)):
                    g = h.graph_of(t)  # raises on any status, the bounds status included
                    o = oracle.compute(f.values, minimum=minimum)
                    ok = (np.array_equal(g.labels, o.label) and np.array_equal(g.maxima, o.maxima)
                          and np.array_equal(g.saddles, o.saddles) and np.array_equal(g.row_ptr, o.row_ptr)
                          and np.array_equal(g.col, o.col) and np.array_equal(g.sad_b0, o.sad_b0))
                    if not ok:
                        print(f"MISMATCH {ext} {kind} minimum={minimum}", flush=True)
                        sys.exit(1)
                    n += 1
    print(f"OK {n}", flush=True)


if __name__ == "__main__":
    main()
