"""Shared helpers for the parity tests (GPU path vs FP64 oracle)."""

import numpy as np

import oracle


def parity_report(osc: "oracle.Scene", o, d, max_range, gpu_range, gpu_id, min_range=0.0):
    """Compare GPU (range, id) per ray with the oracle under the tolerance
    contract; flagged rays must still pass the oracle's plausibility check."""
    gr = np.asarray(gpu_range, np.float32)
    gi = np.asarray(gpu_id, np.int32)
    r_o, i_o, fl = osc.cast(o, d, max_range, min_range=min_range)
    bad, checked = oracle.compare(gr, gi, r_o, i_o, fl, max_range)
    flagged = fl != 0
    invalid = 0
    if flagged.any():
        ok = osc.validate(o[flagged], d[flagged], max_range, gr[flagged], gi[flagged],
                          min_range=min_range)
        invalid = int((~ok).sum())
    return {
        "n": len(gr),
        "bad": int(bad.sum()),
        "bad_idx": np.nonzero(bad)[0][:10].tolist(),
        "flagged": int(flagged.sum()),
        "invalid_flagged": invalid,
        "hits": int((i_o >= 0).sum()),
        "id_mismatch_any": int((gi != i_o).sum()),
        "max_abs_range_err_unflagged": float(np.max(np.abs(gr[~flagged] - r_o[~flagged]), initial=0.0)),
    }


def assert_parity(rep):
    assert rep["bad"] == 0, rep
    assert rep["invalid_flagged"] == 0, rep


def oracle_mesher(gs, origin, h, dims):
    """The 3DGS-to-mesh steps of the oracle (density, denoise, TSDF, marching
    tetrahedra) as a mesher for synth.workloads.hetero_meshes."""
    return oracle.mesh_from_gaussians(gs.mu, gs.scale, gs.quat, gs.alpha, origin, h, dims)
