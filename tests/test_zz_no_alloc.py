"""tc_pressure_map_noalloc: the allocation-free pressure map, for callers that
cannot allocate device memory when they call it (its scratch is a fixed
file-scope device array).  Checked through the C ABI against tc_pressure_map
on the same env, on two calls in a row (the second call reuses the shared
scratch left by the first).  Collected last so that a failure here does not
hide the results of the other GPU tests."""
import numpy as np
import pytest

from gpu_util import rel_fro
from synth import workloads

pytestmark = pytest.mark.gpu


def _tables(env, g):
    """Device inputs of the allocation-free call, built from what the env's
    public calls return (test-side bookkeeping only)."""
    import torch
    faces, parent = g.surface_faces()
    verts = np.unique(faces)
    slot = np.searchsorted(verts, faces).astype(np.int32)          # (nfc, 3)
    inc = [(slot[f, k], f * 4 + k) for f in range(len(faces)) for k in range(3)]
    inc.sort()
    off = np.zeros(len(verts) + 1, dtype=np.int32)
    for s_, _ in inc:
        off[s_ + 1] += 1
    off = np.cumsum(off).astype(np.int32)
    idx = np.array([c for _, c in inc], dtype=np.int32)
    pf, pw = g.pixel_table()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(cfaces=dev(faces.T), cparent=dev(parent), cface_slot=dev(slot.T), cv_face_off=dev(off),
                cv_face_idx=dev(idx), pix_face=dev(pf), pix_w=dev(pw.T))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_pressure_map_matches_env_map(precision):
    import torch
    from paper_2606_20426_gb300 import Env
    from paper_2606_20426_gb300.tacauchy import pressure_map_noalloc
    env = workloads.small_env(0, steps=2)
    g = Env(env, precision=precision)
    tab = _tables(env, g)
    H, W = env["grid"]["H"], env["grid"]["W"]
    for k in range(2):  # two calls in a row, each after a step
        g.step(env["poses"][k])
        ref, ref_mask = g.pressure_map()
        x = torch.from_numpy(np.ascontiguousarray(g.positions().T.astype(np.float32))).cuda()
        sig = g.stress()
        out = torch.full((H * W,), float("nan"), dtype=torch.float32, device="cuda")
        mask = torch.zeros((H * W,), dtype=torch.uint8, device="cuda")
        pressure_map_noalloc(x, sig, tab["cfaces"], tab["cparent"], tab["cface_slot"], tab["cv_face_off"],
                             tab["cv_face_idx"], tab["pix_face"], tab["pix_w"], out, mask)
        r = ref.cpu().numpy().ravel()
        assert np.array_equal(mask.cpu().numpy(), ref_mask.cpu().numpy().ravel())
        assert np.abs(r).max() > 0
        assert rel_fro(out.cpu().numpy(), r) <= 1e-3
    g.close()


def test_noalloc_rejects_oversize():
    from paper_2606_20426_gb300 import tacauchy
    lib = tacauchy.load()
    # more contact faces than the scratch holds
    rc = lib.tc_pressure_map_noalloc(None, 0, None, 0, None, None, None, 262145, None, None, 0,
                                     None, None, 0, None, None, None)
    assert rc == 12  # TC_ERR_CAPACITY
    # more contact vertices than the scratch holds
    rc = lib.tc_pressure_map_noalloc(None, 0, None, 0, None, None, None, 0, None, None, 262145,
                                     None, None, 0, None, None, None)
    assert rc == 12


def test_noalloc_without_contact_faces_gives_zero_map():
    """No contact face and no pixel covered: every value and mask entry is 0,
    whatever the shared scratch held from earlier calls."""
    import torch
    from paper_2606_20426_gb300.tacauchy import pressure_map_noalloc
    npix = 1000
    z32 = torch.zeros((3, 0), dtype=torch.int32, device="cuda")
    x = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    sig = torch.zeros((6, 1), dtype=torch.float32, device="cuda")
    off = torch.zeros((1,), dtype=torch.int32, device="cuda")
    idx = torch.zeros((0,), dtype=torch.int32, device="cuda")
    pix_face = torch.full((npix,), -1, dtype=torch.int32, device="cuda")
    pix_w = torch.full((3, npix), 0.25, dtype=torch.float32, device="cuda")
    out = torch.full((npix,), float("nan"), dtype=torch.float32, device="cuda")
    mask = torch.full((npix,), 7, dtype=torch.uint8, device="cuda")
    pressure_map_noalloc(x, sig, z32, torch.zeros((0,), dtype=torch.int32, device="cuda"), z32, off, idx,
                         pix_face, pix_w, out, mask)
    assert torch.count_nonzero(out).item() == 0 and not torch.isnan(out).any().item()
    assert torch.count_nonzero(mask).item() == 0
