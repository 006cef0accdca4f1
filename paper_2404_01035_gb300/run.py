"""Run a simulation from the paper's input files.

    python -m paper_2404_01035_gb300.run INFILE FILLING [--steps N] [--save-every K]
                                         [--out DIR] [--dtype f32|f64] [--dry-run] ...
    python -m paper_2404_01035_gb300.run INFILE --restart DIR/checkpoint.bin [--steps N] ...

The infile gives the grid and the parameters (`read_infile`), the filling
file the initial phases (`read_filling`).  The initial chemical potential is
uniform, the value at which the liquid has its fill composition (cfill of the
liquid, else its ceq).  Every `--save-every` steps (default SAVET, else
NTIMESTEPS) the driver prints the FP64 diagnostics as one JSON line and
writes the state to DIR/step_<n>.npz (phi, mu, step, t), or with
`--format vtk` to DIR/step_<n>.vtk (legacy VTK, one scalar per phase and
solute).  With `--checkpoint` it also keeps DIR/checkpoint.bin, the
library's checkpoint of the latest saved state (its step and time included);
`--restart` resumes from such a file, bitwise where the run left off, and
steps on to the same total.  A deck with `Shift = 1` runs in the moving frame:
the growth front is kept at index Shiftj of the last axis, and liquid of the
alloy's chemical potential refills the far end.  It stops with exit code 3 if the library reports
a non-finite state.  `--dry-run` reads and
checks the inputs and prints their summary without touching the GPU; the
summary carries the library's own verdict on them (`library_check`) and
the stability bound on dt (`dt_bound`), and a refused deck ends with exit
code 2 before any GPU work.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
from typing import List, Optional

import numpy as np

from .infile import liquid_mu, read_filling, read_infile


def alloy_mu(spec) -> np.ndarray:
    """The uniform chemical potential of the alloy: the liquid at its fill
    composition (cfill), else at its equilibrium composition (ceq)."""
    liq = spec.n_phases - 1
    return liquid_mu(spec, spec.meta["cfill"].get(liq, list(spec.ceq[liq])))


def build_inputs(args):
    spec = read_infile(args.infile, free_energy=args.free_energy, elasticity=args.elasticity,
                       anti_trapping=args.anti_trapping, grain_growth=args.grain_growth,
                       noise_seed=args.noise_seed)
    if args.filling is None:                # a restart: the state comes from the checkpoint
        return spec, None, None
    phi0 = read_filling(args.filling, spec, diffuse=not args.sharp)
    mu0 = np.broadcast_to(alloy_mu(spec)[:, None, None, None], (spec.n_mu,) + phi0.shape[1:]).copy()
    return spec, phi0, mu0


def write_vtk(path: str, phi: np.ndarray, mu: np.ndarray, dx: float, names=None, title: str = "microsim"):
    """Legacy VTK structured points (binary, big-endian FP64), one point per
    cell at its centre: phi_<phase> then mu_<solute> scalars, readable by
    ParaView and VisIt."""
    nz, ny, nx = phi.shape[1:]
    names = names or [f"phi_{a}" for a in range(phi.shape[0])] + [f"mu_{i}" for i in range(mu.shape[0])]
    with open(path, "wb") as f:
        head = (f"# vtk DataFile Version 3.0\n{title}\nBINARY\nDATASET STRUCTURED_POINTS\n"
                f"DIMENSIONS {nx} {ny} {nz}\nORIGIN {dx / 2!r} {dx / 2!r} {dx / 2!r}\n"
                f"SPACING {dx!r} {dx!r} {dx!r}\nPOINT_DATA {nx * ny * nz}\n")
        f.write(head.encode())
        for name, field_ in zip(names, list(phi) + list(mu)):
            f.write(f"SCALARS {name} double 1\nLOOKUP_TABLE default\n".encode())
            f.write(np.ascontiguousarray(field_, dtype=">f8").tobytes())
            f.write(b"\n")


def _summary(spec, phi0, mu0, steps, every):
    return {
        "grid": [spec.dim, spec.nx, spec.ny, spec.nz], "dx": spec.dx, "dt": spec.dt,
        "phases": spec.n_phases, "components": spec.n_components, "bc": list(spec.bc)[: spec.dim],
        "potential": spec.potential, "anisotropic": bool(np.any(spec.delta)),
        "temperature": {"T0": spec.T0, "G": spec.G, "z0": spec.z0, "V": spec.V},
        "options": {"anti_trapping": spec.anti_trapping, "grain_growth": spec.grain_growth,
                    "elasticity": spec.elastic_C is not None, "noise_amp": spec.noise_amp},
        "phase_fractions": None if phi0 is None else [float(v) for v in phi0.reshape(spec.n_phases, -1).mean(axis=1)],
        "mu0": None if mu0 is None else [float(v) for v in mu0.reshape(spec.n_mu, -1)[:, 0]],
        "moving_frame": {"on": bool(spec.meta["shift"]), "keep": spec.meta["shiftj"]},
        "steps": steps, "save_every": every, "ignored_keys": spec.meta["ignored"],
    }


def main(argv: Optional[List[str]] = None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2404_01035_gb300.run", description=__doc__.split("\n\n")[0])
    ap.add_argument("infile")
    ap.add_argument("filling", nargs="?", default=None)
    ap.add_argument("--steps", type=int, default=None, help="default: NTIMESTEPS")
    ap.add_argument("--save-every", type=int, default=None, help="default: SAVET, else the whole run")
    ap.add_argument("--out", default="microsim_out")
    ap.add_argument("--format", choices=("npz", "vtk"), default="npz", help="snapshot format")
    ap.add_argument("--dtype", choices=("f32", "f64"), default="f32")
    ap.add_argument("--sharp", action="store_true", help="fill shapes without the equilibrium profile")
    ap.add_argument("--free-energy", choices=("parabolic",), default=None)
    ap.add_argument("--elasticity", action="store_true")
    ap.add_argument("--anti-trapping", action="store_true")
    ap.add_argument("--grain-growth", action="store_true")
    ap.add_argument("--noise-seed", type=int, default=0)
    ap.add_argument("--checkpoint", action="store_true", help="keep DIR/checkpoint.bin of the latest save")
    ap.add_argument("--restart", default=None, help="resume from a checkpoint file")
    ap.add_argument("--dry-run", action="store_true")
    args = ap.parse_args(argv)
    if (args.filling is None) == (args.restart is None):
        ap.error("give a FILLING file for a new run or --restart CHECKPOINT to resume one")

    spec, phi0, mu0 = build_inputs(args)
    steps = args.steps if args.steps is not None else spec.steps
    if steps < 0:
        ap.error("--steps must be >= 0")
    if args.save_every is not None and args.save_every <= 0:
        ap.error("--save-every must be > 0")
    every = args.save_every or spec.meta.get("savet") or steps or 1
    info = _summary(spec, phi0, mu0, steps, every)
    # the library's own checks (inputs, derived coefficients, compiled kernels,
    # dt against the stability bound), on the host: no GPU is touched
    from ._binding import MSError
    from .simulation import check_params
    try:
        info["dt_bound"] = check_params(spec, args.dtype)
        info["library_check"] = "ok"
    except MSError as e:
        info["dt_bound"] = getattr(e, "dt_bound", None)
        info["library_check"] = str(e)
    print(json.dumps({"inputs": info}), flush=True)
    if info["library_check"] != "ok":
        return 2
    if args.dry_run:
        return 0

    from .simulation import Simulation      # needs the CUDA library and a GPU
    os.makedirs(args.out, exist_ok=True)

    names = ([f"phi_{n}" for n in spec.meta["phases"]] if len(spec.meta["phases"]) == spec.n_phases
             else [f"phi_{a}" for a in range(spec.n_phases)]) + [f"mu_{i}" for i in range(spec.n_mu)]

    def save(sim, d):
        if args.checkpoint:
            tmp = os.path.join(args.out, "checkpoint.bin.tmp")
            with open(tmp, "wb") as f:
                f.write(sim.checkpoint())
            os.replace(tmp, os.path.join(args.out, "checkpoint.bin"))
        phi, mu = sim.get_fields()
        stem = os.path.join(args.out, f"step_{d['step']:010d}")
        if args.format == "vtk":
            write_vtk(stem + ".vtk", phi, mu, spec.dx, names, f"step {d['step']} t {d['t']!r}")
        else:
            np.savez(stem + ".npz", phi=phi, mu=mu, step=d["step"], t=d["t"])

    with Simulation(spec, dtype=args.dtype) as sim:
        if args.restart:
            with open(args.restart, "rb") as f:
                sim.restore(f.read())
            d = sim.diag()
        else:
            sim.set_fields(phi0, mu0)
            d = sim.diag()
            save(sim, d)
        done = int(d["step"])
        while done < steps:
            k = min(every, steps - done)
            try:
                if spec.meta["shift"]:
                    # SHIFT: keep the growth front at index Shiftj of the last axis,
                    # refilling the far end with liquid of the alloy's mu
                    sim.step_moving_frame(k, keep=spec.meta["shiftj"], mu_fill=alloy_mu(spec),
                                          check_every=min(100, k))
                else:
                    sim.step(k)
                d = sim.diag()
            except MSError as e:
                if e.status != 5:               # anything but MS_ERR_NONFINITE
                    raise
                print(json.dumps({"error": "the state became non-finite", "after_step": done + k}), flush=True)
                return 3
            done += k
            print(json.dumps({"step": d["step"], "t": d["t"], "mass": [float(v) for v in d["mass"]],
                              "sum_err": d["sum_err"], "phi_min": d["phi_min"], "phi_max": d["phi_max"]}),
                  flush=True)
            save(sim, d)
    return 0


if __name__ == "__main__":
    sys.exit(main())
