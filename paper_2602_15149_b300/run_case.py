"""Run one of the synthetic workloads for a number of steps and report the time per step.

    python -m paper_2602_15149_b300.run_case crack_branching --nx 400 --steps 200
    python -m paper_2602_15149_b300.run_case flyer_plate --n 50 --steps 500 --mode graph

The workload is built by paper_2602_15149_b300.workloads with the given size, stepped through the C-ABI
after a few warm-up steps, and timed with CUDA events on the context's stream.
"""
from __future__ import annotations

import argparse
import json

from . import tlsph, workloads as W

CASES = {
    "block_3d": lambda a: W.block_3d(nx=a.nx or 128, ny=a.ny or 128, nz=a.nz or 64),
    "plate_2d": lambda a: W.plate_2d(nx=a.nx or 100, ny=a.ny or 20),
    "notched_plate": lambda a: W.notched_plate(nx=a.nx or 500, ny=a.ny or 200, model=a.model or "nh"),
    "crack_branching": lambda a: W.crack_branching(nx=a.nx or 1600, ny=(a.nx or 1600) * 2 // 5),
    "cantilever_beam": lambda a: W.cantilever_beam(dx=a.dx or 0.5e-3, precision="fp32"),
    "flyer_plate": lambda a: W.flyer_plate(n=a.n or 100),
    "taylor_bar": lambda a: W.taylor_bar(dx=a.dx or 0.4e-3),
}
MODES = {"launch": tlsph.MODE_LAUNCH, "graph": tlsph.MODE_GRAPH, "persistent": tlsph.MODE_PERSISTENT}
LAYOUTS = {"auto": tlsph.LAYOUT_AUTO, "csr": tlsph.LAYOUT_CSR}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--nx", type=int)
    ap.add_argument("--ny", type=int)
    ap.add_argument("--nz", type=int)
    ap.add_argument("--n", type=int)
    ap.add_argument("--dx", type=float)
    ap.add_argument("--model", choices=["nh", "svk"])
    ap.add_argument("--mode", choices=sorted(MODES), default="launch")
    ap.add_argument("--layout", choices=sorted(LAYOUTS), default="auto")
    a = ap.parse_args(argv)
    import torch

    case = CASES[a.case](a)
    stream = torch.cuda.Stream(device=0)
    g = tlsph.from_case(case, stream=stream.cuda_stream)
    g.set_option(tlsph.OPT_MODE, MODES[a.mode])
    g.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, LAYOUTS[a.layout])
    g.step(a.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step_async(a.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    status = g.sync(check=False)
    ms = e0.elapsed_time(e1) / max(a.steps, 1)
    info = g.get_info()
    print(json.dumps({"case": case.name, "particles": case.n, "steps": a.steps, "ms_per_step": ms,
                      "particle_steps_per_s": case.n / (ms * 1e-3), "status": int(status),
                      "kernel_launches": info["kernel_launches"], "neighbour_pairs": info["nnz"],
                      "layout": a.layout, "stencil_entries": info["stencil"]}))
    g.close()
    return 0 if status == tlsph.OK else 1


if __name__ == "__main__":
    raise SystemExit(main())
