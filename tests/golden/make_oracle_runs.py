"""Write the FP64 oracle's whole-run references that the GPU parity tests read.

Test infrastructure: this script calls only the oracle (``oracle/``) and the
seeded input generators (``paper_2003_12693_gb300/synth.py``); nothing in its
output comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_oracle_runs.py [config ...]

For each configuration it runs Alg. 1 three times in FP64 from inputs rounded
to FP32 (the numbers the GPU receives):

  ref   the inputs as given;
  T     the inputs transposed (every operator of the method is symmetric
        under swapping the axes, so in exact arithmetic this is ref^T);
  P     the inputs perturbed by one FP32 unit in the last place (a seeded
        random choice of -1, 0, +1 ulp per pixel of the image and of phi0).

T and P measure how strongly the method itself amplifies rounding: T a
change of summation order only, P a change of the data at FP32 accuracy
(what an FP32 implementation commits in its first operation).  Recorded per
checkpoint: max|phi_ref - phi_T^T| and max|phi_ref - phi_P|, mask
disagreements, the {phi < 0} component count (4-connected) and the discrete
energy of Eqs. (7)-(10).  Stored at the last checkpoint: the three masks and
the pixels where |phi_ref| < 1e-3.

A second set, ``early``, uses a tie-free initial rectangle (edges offset by a
quarter and a half pixel, so that no pixel lies on a ridge of the signed
distance where forward differences vanish and w = B/|B| would take the
direction of rounding noise) and records the same sensitivities for every
iteration until the P difference passes 1e-4; the GPU test of the early
iterations runs to the last K whose P difference is <= 2e-5, a fifth of the
1e-4 tolerance on phi.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2003_12693_gb300 import synth  # noqa: E402

# name: (workload, crop origin or None, K, checkpoint every)
CONFIGS = {
    "two_disks_128": ("two_disks_128", None, 200, 10),
    "ellipses_512": ("ellipses_512", None, 1000, 50),
    "blobs_4096_crop512": ("blobs_4096", (1792, 1792), 2000, 100),
}
# early-iteration sets: (workload, crop origin or None, iteration cap)
EARLY = {
    "two_disks_128": ("two_disks_128", None, 40),
    "ellipses_512": ("ellipses_512", None, 40),
    "ellipses_2048": ("ellipses_2048", None, 12),
    "blobs_4096_crop512": ("blobs_4096", (1792, 1792), 40),
}
CROP = 512


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def inputs(workload: str, crop):
    wl = synth.WORKLOADS[workload]
    f = wl.image()
    phi0 = wl.phi0()
    if crop is not None:
        i0, j0 = crop
        f = np.ascontiguousarray(f[i0:i0 + CROP, j0:j0 + CROP])
        phi0 = synth.inset_rect_sdf(CROP, CROP)
    return f32(f), f32(phi0), oracle.Params.from_dict(wl.params())


def tie_free_phi0(workload: str, H: int, W: int):
    """The workload's rectangle with its four edges moved by 1/4, 1/2, 0 and
    1/4 pixel: r0 - c0, r0 + c1, r1 + c0, r1 - c1 and the two mid-lines are
    then never integers, so no pixel is equidistant from two edges."""
    if workload == "two_disks_128":
        r0, r1, c0, c1 = 36, 92, 14, 114
    else:
        r0, r1, c0, c1 = 8, H - 9, 8, W - 9
    return f32(synth.rect_sdf(H, W, r0 + 0.25, r1 + 0.5, c0, c1 + 0.25))


def perturb(a, rng):
    ulp = np.spacing(np.abs(a).astype(np.float32)).astype(np.float64)
    return f32(a + ulp * rng.choice([-1.0, 0.0, 1.0], a.shape))


def components(phi) -> int:
    from scipy import ndimage
    return int(ndimage.label(phi < 0)[1])


def three_runs(f, phi0, p, seed=0):
    rng = np.random.default_rng(seed)
    fP, phi0P = perturb(f, rng), perturb(phi0, rng)
    runs = {}
    for key, (ff, pp) in {"ref": (f, phi0), "T": (f.T.copy(), phi0.T.copy()),
                          "P": (fP, phi0P)}.items():
        runs[key] = (oracle.edge(ff), oracle.initial_state(pp))
    return runs


def whole_run(name: str) -> None:
    workload, crop, K, every = CONFIGS[name]
    f, phi0, p = inputs(workload, crop)
    runs = three_runs(f, phi0, p)
    g_ref = runs["ref"][0]
    trace = {"k": [], "dphi_T": [], "dphi_P": [], "mask_T": [], "mask_P": [],
             "components": [], "components_P": [], "energy": [], "energy_P": []}
    trace["k"].append(0)
    trace["dphi_T"].append(0.0)
    trace["dphi_P"].append(0.0)
    trace["mask_T"].append(0)
    trace["mask_P"].append(0)
    trace["components"].append(components(phi0))
    trace["components_P"].append(components(phi0))
    trace["energy"].append(float(oracle.energy(phi0, g_ref, p)[0]))
    trace["energy_P"].append(trace["energy"][0])
    t0 = time.time()
    for k in range(every, K + 1, every):
        for key in runs:
            oracle.iterate(runs[key][1], runs[key][0], every, p)
        a = runs["ref"][1].phi
        b = runs["T"][1].phi.T
        c = runs["P"][1].phi
        trace["k"].append(k)
        trace["dphi_T"].append(float(np.abs(a - b).max()))
        trace["dphi_P"].append(float(np.abs(a - c).max()))
        trace["mask_T"].append(int(((a < 0) != (b < 0)).sum()))
        trace["mask_P"].append(int(((a < 0) != (c < 0)).sum()))
        trace["components"].append(components(a))
        trace["components_P"].append(components(c))
        trace["energy"].append(float(oracle.energy(a, g_ref, p)[0]))
        trace["energy_P"].append(float(oracle.energy(c, g_ref, p)[0]))
        print(f"{name} k={k} dT={trace['dphi_T'][-1]:.3g} dP={trace['dphi_P'][-1]:.3g} "
              f"mask T/P={trace['mask_T'][-1]}/{trace['mask_P'][-1]} "
              f"comp={trace['components'][-1]} E={trace['energy'][-1]:.6g} "
              f"({time.time() - t0:.0f} s)", flush=True)
    a = runs["ref"][1].phi
    np.savez_compressed(
        os.path.join(HERE, f"whole_run_{name}.npz"),
        mask_ref=np.packbits(a < 0), mask_T=np.packbits(runs["T"][1].phi.T < 0),
        mask_P=np.packbits(runs["P"][1].phi < 0), near_zero=np.packbits(np.abs(a) < 1e-3),
        shape=np.array(a.shape), K=np.array(K))
    meta = {"workload": workload, "crop": crop, "K": K, "trace": trace,
            "how": "tests/golden/make_oracle_runs.py (FP64 oracle only)"}
    with open(os.path.join(HERE, f"whole_run_{name}.json"), "w") as fh:
        json.dump(meta, fh, indent=1)


def early(name: str) -> dict:
    workload, crop, cap = EARLY[name]
    f, _, p = inputs(workload, crop)
    H, W = f.shape
    phi0 = tie_free_phi0(workload, H, W)
    runs = three_runs(f, phi0, p, seed=1)
    dT, dP = [], []
    for k in range(1, cap + 1):
        for key in runs:
            oracle.iterate(runs[key][1], runs[key][0], 1, p)
        a = runs["ref"][1].phi
        dT.append(float(np.abs(a - runs["T"][1].phi.T).max()))
        dP.append(float(np.abs(a - runs["P"][1].phi).max()))
        print(f"early {name} k={k} dT={dT[-1]:.3g} dP={dP[-1]:.3g}", flush=True)
        if dP[-1] > 1e-4:
            break
    K = 0
    for d in dP:  # the last K before the first one above 2e-5
        if d > 2e-5:
            break
        K += 1
    return {"workload": workload, "crop": crop, "phi0": "tie-free rectangle (see tie_free_phi0)",
            "dphi_T": dT, "dphi_P": dP, "K": K}


def main(argv):
    names = argv or list(CONFIGS) + ["early"]
    for name in names:
        if name == "early":
            out = {n: early(n) for n in EARLY}
            with open(os.path.join(HERE, "early_iterations.json"), "w") as fh:
                json.dump(out, fh, indent=1)
        else:
            whole_run(name)


if __name__ == "__main__":
    main(sys.argv[1:])
