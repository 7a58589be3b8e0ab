"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare element by element."""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc

DISP_ATOL = 1e-4    # px, sub-pixel disparity
DEPTH_RTOL = 1e-5   # relative, depth

INT_BLOCK_FIELDS = ("n_pts", "n_valid", "d_f", "dy_f", "d_b", "dy_b", "s_m", "s_0", "s_p", "flags")


def torch_frames(frames, device="cuda"):
    import torch
    return [(torch.from_numpy(np.ascontiguousarray(f.left)).to(device),
             torch.from_numpy(np.ascontiguousarray(f.right)).to(device)) for f in frames]


def compare_box_outputs(got, ref, where=""):
    gf = np.asarray(got["flags"]).astype(np.uint8)
    rf = np.asarray(ref["flags"]).astype(np.uint8)
    bad = np.nonzero(gf != rf)[0]
    assert bad.size == 0, f"{where} flags differ at {bad[:10]}: gpu {gf[bad[:10]]} oracle {rf[bad[:10]]}"
    gd, rd = np.asarray(got["disp"]), np.asarray(ref["disp"])
    assert np.array_equal(np.isnan(gd), np.isnan(rd)), where
    ok = ~np.isnan(rd)
    np.testing.assert_allclose(gd[ok], rd[ok], rtol=0, atol=DISP_ATOL, err_msg=where)
    gz, rz = np.asarray(got["depth"]), np.asarray(ref["depth"])
    assert np.array_equal(np.isnan(gz), np.isnan(rz)), where
    okz = ~np.isnan(rz)
    np.testing.assert_allclose(gz[okz], rz[okz], rtol=DEPTH_RTOL, atol=0, err_msg=where)


def compare_debug(dbg, ref, nc_gpu, where=""):
    compare_debug_arrays(dbg.blocks_np(), dbg.cost_f.cpu().numpy(), dbg.cost_b.cpu().numpy(), ref,
                         nc_gpu, where)


def compare_debug_arrays(gb, gcf, gcb, ref, nc_gpu, where=""):
    rb = ref["blocks"]
    assert gb.shape == rb.shape, (gb.shape, rb.shape)
    for f in INT_BLOCK_FIELDS:
        bad = np.argwhere(gb[f] != rb[f])
        assert bad.size == 0, f"{where} block field {f} differs at {bad[:5].tolist()}: " \
                              f"gpu {gb[f][tuple(bad[0])]} oracle {rb[f][tuple(bad[0])]}"
    for f in ("d_sub", "d_full"):
        np.testing.assert_allclose(gb[f], rb[f], rtol=0, atol=DISP_ATOL, err_msg=f"{where} {f}")
    nc = min(nc_gpu, ref["cost_f"].shape[2])
    assert np.array_equal(gcf[..., :nc], ref["cost_f"][..., :nc]), f"{where} forward costs differ"
    assert np.array_equal(gcb[..., :nc], ref["cost_b"][..., :nc]), f"{where} backward costs differ"


def oracle_evals(ref_blocks, boxes_flags, params: dict) -> int:
    """Cost evaluations implied by the oracle's blocks: 2 * n_valid * NC per searched block."""
    ndy = params["dy_max"] - params["dy_min"] + 1
    nd_far = params["far_dmax"] - params["far_dmin"] + 1
    nd_close = params["close_dmax"] - params["close_dmin"] + 1
    total = 0
    for i in range(ref_blocks.shape[0]):
        far = bool(boxes_flags[i] & orc.BOX_FAR)
        nc = (nd_far if far else nd_close) * ndy
        for b in ref_blocks[i]:
            if (b["flags"] & orc.BLK_PRESENT) and not (b["flags"] & orc.BLK_FEW_POINTS):
                total += 2 * int(b["n_valid"]) * nc
    return total
