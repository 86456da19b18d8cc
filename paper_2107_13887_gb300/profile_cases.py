"""Small cases of the library's main kernels, for profiler captures.

Each case runs the hot path once on inputs a profiler can replay in a few
seconds (a few hundred MB on the device, larger than L2 where the kernel's
DRAM traffic matters), the same kernels as the benchmark's workloads:

    python -m paper_2107_13887_gb300.profile_cases persist    # k_greedy_persist, k_greedy_newton, k_vol_sweep_f32
    python -m paper_2107_13887_gb300.profile_cases worklist   # k_vol_worklist over four uneven wings
    python -m paper_2107_13887_gb300.profile_cases persist_mid  # k_greedy_persist, 304 blocks

persist:  the swept wing of the benchmark at 1/15 of its surface (100 x 40 =
          4,000 points, 400k volume points), its three levels to 1e-5 in the
          persistent list sweep alone (engine 2: at this size the Newton
          start would take every level; on the 60k wing it hands levels 1
          and 2 to this launch), then the volume update.
persist_mid: the swept wing at a quarter of the benchmark's surface (200 x
          75 = 15,000 points), the three levels in the persistent list sweep
          alone with at most 6,000 controls per level (G and G^T 0.6 GB):
          the third launch (R = 0.1, 6,000 steps) runs 304 blocks (118 point
          blocks) with G rows of up to 6,000 entries.
worklist: the four-wing family at 1/25 of its surfaces (1.2k to 10k points)
          and 60 layers (72k to 600k volume points each, 1.2M in all), two
          levels to 1e-3, the volume updates of all four in one work-list
          launch with fixed settings (R / 2 cells, 8 blocks per SM).
"""
from __future__ import annotations

import sys

import numpy as np

from . import rbfd, synth


def run_persist():
    c = synth.wing_case(100, 40, 100, displacement="ridge", seed=0, R=(1.5, 0.4, 0.1), eps=1e-5, D=1.0, k=4.0)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, engine=2)
    m.greedy()
    out = m.deform(c.xyz_v, c.d_v, c.D, c.k)
    st = m.stats()
    print(f"persist case: controls {[len(L.idx) for L in m.levels()]}, greedy {st['greedy_ms']:.1f} ms, "
          f"deform {st['deform_ms']:.2f} ms, finite {bool(np.isfinite(out).all())}")
    m.close()


def run_persist_mid():
    c = synth.wing_case(200, 75, 2, displacement="ridge", seed=0, R=(1.5, 0.4, 0.1), eps=1e-5, D=1.0, k=4.0,
                        wall_distance=False)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, engine=2, nc_cap=6000)
    rc = m.greedy()
    st = m.stats()
    print(f"persist_mid case: status {rc}, controls {[len(L.idx) for L in m.levels()]}, "
          f"greedy {st['greedy_ms']:.1f} ms")
    m.close()


def run_worklist():
    cases = [synth.wing_case(nc, ns, 60, displacement="ridge", seed=s, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0)
             for s, (nc, ns) in enumerate([(40, 30), (80, 40), (100, 60), (125, 80)])]
    ms = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps) for c in cases]
    rbfd.greedy_batch(ms)
    outs = [np.empty((c.n_v, 3), np.float32) for c in cases]
    t = rbfd.deform_worklist(ms, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                             [c.k for c in cases], outs, autotune=False, ctas_per_sm=8, item_blocks=1,
                             cell_div=[2, 2, 2, 2])
    print(f"worklist case: volume points {[c.n_v for c in cases]}, launch {t['launch_ms']:.2f} ms, "
          f"items {t['items']}")
    for m in ms:
        m.close()


def main(argv):
    which = argv[1] if len(argv) > 1 else "persist"
    {"persist": run_persist, "persist_mid": run_persist_mid, "worklist": run_worklist}[which]()


if __name__ == "__main__":
    main(sys.argv)
