"""CPU-side checks of the C ABI: the library builds, loads, exports every declared
symbol, and validates arguments on the host (no GPU work is issued)."""
import ctypes

import numpy as np
import pytest

import paper_2604_27158_gb300 as P
from paper_2604_27158_gb300 import _abi
from paper_2604_27158_gb300.lbm import GridSpec, query_layout


def test_library_exports_every_declared_symbol():
    lib = P.lib()
    names = _abi.declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_query_layout_sizes():
    grids = [GridSpec(128, 64, 0.8), GridSpec(37, 20, 0.6, bc_west=P.BC_PRESSURE,
                                                bc_east=P.BC_PRESSURE, west_value=1.001)]
    lay = query_layout(grids)
    assert lay.cells == 128 * 64 + 37 * 20
    assert lay.f_elems == 9 * (64 * 128 + 20 * 64)       # pitch = nx rounded up to 32
    assert lay.mask_words == 64 * 4 + 20 * 2
    assert lay.ws_bytes > 0 and lay.ws_bytes % 256 == 0


@pytest.mark.parametrize("bad", [
    GridSpec(1, 8, 0.8),                                   # too small
    GridSpec(8, 8, 0.5),                                   # tau must exceed 1/2
    GridSpec(8, 8, 0.8, bc_west=P.BC_PRESSURE),            # periodic on one end only
    GridSpec(8, 8, 0.8, bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE, west_value=0.7),
    GridSpec(8, 8, 0.8, bc_west=7, bc_east=7),
])
def test_query_layout_rejects_invalid_grids(bad):
    with pytest.raises(P.LbmError) as e:
        query_layout([bad])
    assert e.value.code == _abi.LBM_ERR_INVALID_ARG
    assert "lbm" in str(e.value)


def test_null_arguments_rejected_without_gpu():
    lib = P.lib()
    assert lib.lbm_query_layout(None, 0, None) == _abi.LBM_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.lbm_init(None, 0, None, None, None, None, 0.2, None, ctypes.byref(h)) == _abi.LBM_ERR_INVALID_ARG
    assert lib.lbm_step(None, 1, None) == _abi.LBM_ERR_INVALID_ARG
    assert h.value is None


def test_mask_packing_layout():
    solid = np.zeros((3, 40), bool)
    solid[1, 33] = True
    solid[2, 0] = True
    w = P.pack_mask(solid)
    assert w.shape == (6,)
    assert w[1 * 2 + 1] == (1 << 1) and w[2 * 2] == 1 and w.sum() == 3


def test_fno_query_counts_the_papers_parameters():
    """The library's parameter layout (fno_query, host only) has exactly the totals the
    paper prints for its six model shapes."""
    import json
    import os
    from paper_2604_27158_gb300.fno import FnoShape, fno_query
    with open(os.path.join(os.path.dirname(__file__), "golden", "fno_param_counts.json")) as fh:
        models = json.load(fh)["models"]
    for mdl in models:
        shape = FnoShape(c_in=mdl["c_in"], c_out=mdl["c_out"], width=mdl["width"],
                         layers=mdl["layers"], modes=mdl["modes"], dec_layers=mdl["dec_layers"],
                         dec_size=mdl["dec_size"])
        sz = fno_query(shape, 1, 2 * mdl["modes"], 2 * mdl["modes"] + 1)
        assert sz.n_params == mdl["params"], mdl["name"]
        assert sz.packed_bytes % 256 == 0 and sz.ws_bytes > 0


@pytest.mark.parametrize("kw,B,H,W", [
    (dict(modes=8), 1, 15, 64),      # 2m > H
    (dict(modes=8), 1, 32, 16),      # m >= W / 2
    (dict(width=15), 1, 32, 32),     # odd width
    (dict(width=66), 1, 32, 32),     # width above 64
    (dict(activation=5), 1, 32, 32),
])
def test_fno_query_rejects_invalid_shapes(kw, B, H, W):
    from paper_2604_27158_gb300.fno import FnoShape, fno_query
    with pytest.raises(P.LbmError) as e:
        fno_query(FnoShape(**kw), B, H, W)
    assert e.value.code == _abi.LBM_ERR_INVALID_ARG


def test_hybrid_workspace_holds_every_group_and_network():
    """An FNO step runs its size groups, and the two networks of a group, as parallel
    branches, so no two of them may share FNO buffers: the hybrid workspace (a host-only
    query) grows by at least the FNO workspaces of both networks when a size group is
    added, and holds those of every (group, network) pair."""
    from paper_2604_27158_gb300._abi import call, lbm_grid
    from paper_2604_27158_gb300.fno import FnoShape, fno_query
    sr = FnoShape(c_in=1, c_out=1, width=16, layers=2, modes=4, dec_size=32)
    su = FnoShape(c_in=2, c_out=2, width=16, layers=2, modes=8, dec_size=32)

    def ws(grids):
        arr = (lbm_grid * len(grids))(*[g.c() for g in grids])
        n = ctypes.c_size_t()
        fc, fcu = sr.c(), su.c()
        call("hybrid_query_ws", arr, len(grids), ctypes.byref(fc), ctypes.byref(fcu),
             ctypes.byref(n))
        return n.value

    one = [GridSpec(128, 64, 0.8)] * 3
    two = one + [GridSpec(96, 48, 0.7)] * 2
    fno_ws = {(B, H, W): fno_query(sr, B, H, W).ws_bytes + fno_query(su, B, H, W).ws_bytes
              for B, H, W in ((3, 64, 128), (2, 48, 96))}
    assert ws(one) >= fno_ws[(3, 64, 128)]
    assert ws(two) - ws(one) >= fno_ws[(2, 48, 96)]
    assert ws(two) >= sum(fno_ws.values())
