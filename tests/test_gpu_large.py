"""The large-mesh kernels (256^3 two-stage, 512^3 and 1024^3 fused x-y passes) at full size.

- Planar slabs: particles sit on cell nodes filling whole x-, y- and z-planes (exactly N_p^3 of
  them), so the density is an exact integer pattern that varies along one axis per slab set. The
  force is then exactly the sum of three 1-D solutions (oracle planar_force_1d), at any mesh size.
- Engines: on a clustered state the default two-stage passes (blocked layout, two-base force
  form), the fused x-y passes and the Stockham engine agree to FP32 rounding.
- 256^3: the oracle's full 3-D force (numpy FFT primitive) on a clustered state.
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_1506_03737_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1506_03737_gb300 import colapm
    return colapm, torch


def planar_state(np_, nm, seed):
    """Cells and zero offsets of N_p^3 particles on the nodes of nm/8 planes (x, y and z sets)."""
    rng = np.random.default_rng(seed)
    nplanes = nm ** 3 // 8 // nm ** 2                      # = nm / 8 when nm = 2 np
    assert nplanes * nm * nm == np_ ** 3
    counts = [nplanes // 3 + (1 if i < nplanes % 3 else 0) for i in range(3)]
    sets = [np.sort(rng.choice(nm, size=c, replace=False)) for c in counts]
    a, b = np.meshgrid(np.arange(nm, dtype=np.int32), np.arange(nm, dtype=np.int32), indexing="ij")
    a, b = a.ravel(), b.ravel()
    cells = []
    for axis, planes in enumerate(sets):
        for p in planes:
            c = np.empty((nm * nm, 3), np.int32)
            c[:, axis] = p
            others = [j for j in range(3) if j != axis]
            c[:, others[0]] = a
            c[:, others[1]] = b
            cells.append(c)
    cell = np.concatenate(cells)
    return cell, np.zeros(cell.shape, np.float32), sets


@pytest.mark.parametrize("np_,nm", [(256, 512), (512, 1024)])
def test_planar_slabs_force_full_size(env, np_, nm):
    C, torch = env
    box = float(nm)
    p = C.default_params(np=np_, nm=nm, box=box, deconv=1)
    ctx = C.colapm_create(p)
    try:
        C.colapm_make_ics(ctx)
        cell, off, sets = planar_state(np_, nm, 17)
        C.colapm_set_state(ctx, cell, off, None)
        f = torch.empty(3 * nm ** 3, dtype=torch.float32, device="cuda")
        C.colapm_get_force(ctx, f)
        f = f.view(3, nm, nm, nm)
        ratio3 = (nm / np_) ** 3
        for axis in range(3):
            d1 = np.zeros(nm)
            d1[sets[axis]] = ratio3                        # one particle per cell on the plane
            ref = opm.planar_force_1d(d1, box, 1) * (nm / box)
            shape = [1, 1, 1]
            shape[2 - axis] = nm                           # mesh is [z][y][x]
            want = torch.from_numpy(ref.reshape(shape)).to("cuda", torch.float64)
            got = f[axis].double()
            err = torch.sqrt(torch.mean((got - want) ** 2)).item()
            assert err < 1e-4 * float(np.sqrt(np.mean(ref ** 2))), axis
    finally:
        C.colapm_destroy(ctx)


def test_engines_agree_at_1024(env):
    C, torch = env
    np_, nm = 512, 1024
    p = C.default_params(np=np_, nm=nm, box=1024.0)
    ctx = C.colapm_create(p)
    try:
        C.colapm_make_ics(ctx)
        cell, off, _ = workloads.clustered_state(np_, nm, 5)
        C.colapm_set_state(ctx, cell, off, None)
        del cell, off
        out = {}
        for name, (fused, two) in {"fused": (3, 1), "two_stage": (0, 1), "stockham": (0, 0)}.items():
            C.colapm_set_engine(ctx, fused, two, 256)
            f = torch.empty(3 * nm ** 3, dtype=torch.float32, device="cuda")
            C.colapm_get_force(ctx, f)
            out[name] = f
        ref = out["two_stage"].double()
        scale = torch.sqrt(torch.mean(ref ** 2)).item()
        for name in ("fused", "stockham"):
            diff = out[name].double() - ref
            assert torch.sqrt(torch.mean(diff ** 2)).item() < 1e-5 * scale, name
    finally:
        C.colapm_destroy(ctx)


def test_force_256_matches_oracle(env):
    C, torch = env
    np_, nm, box = 128, 256, 300.0
    ctx = C.colapm_create(C.default_params(np=np_, nm=nm, box=box))
    try:
        C.colapm_make_ics(ctx)
        cell, off, _ = workloads.clustered_state(np_, nm, 3)
        C.colapm_set_state(ctx, cell, off, None)
        f = np.empty(3 * nm ** 3, np.float32)
        C.colapm_get_force(ctx, f)
        f = f.reshape(3, nm, nm, nm)
        rho = opm.cic_deposit(cell.astype(np.float64) + off, nm)
        ref = opm.force_mesh(opm.density_contrast(rho, np_, nm), box, 1, fft="numpy") * (nm / box)
        for j in range(3):
            err = np.sqrt(np.mean((f[j].astype(np.float64) - ref[j]) ** 2)) / np.sqrt(np.mean(ref[j] ** 2))
            assert err < 1e-4, j
    finally:
        C.colapm_destroy(ctx)
