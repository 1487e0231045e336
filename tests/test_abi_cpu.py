"""The C ABI on a machine without a GPU: the library loads, exports every
function include/ccell.h declares, and its host-only queries (grid, stepped
outline, status strings) agree with the oracle's grid and outline."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle
from paper_1408_5853_gb300 import ccell, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccell.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)  # drop comments
    text = re.sub(r"//[^\n]*", " ", text)
    return sorted(set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    names = declared_functions()
    assert len(names) >= 15, names
    lib = ctypes.CDLL(ccell.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    for code in range(0, -9, -1):
        s = ccell.cc_status_string(code)
        assert s and "unknown" not in s.lower(), (code, s)


@pytest.mark.parametrize("case", ["small", "production", "paper"])
def test_host_grid_matches_oracle_grid(case):
    cfg = {"small": inputs.small_case(q0=1.0), "production": inputs.production_case(),
           "paper": inputs.paper_case(128, 301)}[case]
    r, z, cls = ccell.cc_query_grid(ccell.geometry_desc(cfg))
    g = oracle.grid(cfg)
    np.testing.assert_allclose(r, g["r"], rtol=1e-15, atol=0.0)
    np.testing.assert_allclose(z, g["z"], rtol=1e-15, atol=0.0)
    assert np.array_equal(np.asarray(cls), g["rclass"])


@pytest.mark.parametrize("layers,z_step", [(1, 4e-3), (2, 6e-3), (3, 9.99e-3), (1, 20e-3)])
def test_host_outline_matches_oracle_outline(layers, z_step):
    cfg = inputs.small_case(q0=1.0)
    cfg["step"] = dict(layers=layers, z=z_step)
    assert ccell.cc_query_outline(ccell.geometry_desc(cfg)) == oracle.outline(cfg)


def test_outline_rejections():
    cfg = inputs.small_case(q0=1.0)
    for step in (dict(layers=4, z=5e-3),       # as many layers as the cylinder
                 dict(layers=1, z=0.01e-3),    # line 1 would be narrow
                 dict(layers=-1, z=5e-3)):
        cfg["step"] = step
        with pytest.raises(ccell.CCError):
            ccell.cc_query_outline(ccell.geometry_desc(cfg))
        with pytest.raises(ValueError):
            oracle.outline(cfg)


@pytest.mark.parametrize("case", ["small", "production", "paper"])
def test_host_stability_bound_matches_oracle(case):
    """cc_tau_stab (host side of the guard of Eq. (stability_condition)) equals
    the oracle's bound over the same temperature range."""
    cfg = {"small": inputs.small_case(q0=1.0), "production": inputs.production_case(),
           "paper": inputs.paper_case(128, 301)}[case]
    lo, hi = (4.2, 20.0) if case == "paper" else (cfg["t_dirichlet"], 100.0)
    cfg["t_guard"] = (lo, hi)
    sol = ccell.Solver(cfg)          # no device work until the first step
    try:
        got = sol.tau_stab(0)
    finally:
        sol.close()
    want = oracle.tau_stab(cfg, lo, hi, 257)
    assert abs(got - want) <= 1e-12 * want, (got, want)


def test_descriptor_and_material_validation():
    cfg = inputs.small_case(q0=1.0)
    bad_descs = []
    for field, value in (("nr", 2), ("nz", 2), ("nr", 513), ("length_m", -1.0),
                         ("bc_rmax", 2), ("placement", 1), ("face_rule", 3)):
        d = ccell.geometry_desc(cfg)
        setattr(d, field, value)
        bad_descs.append((field, d))
    for field, d in bad_descs:
        with pytest.raises(ccell.CCError):
            ccell.cc_create_geometry([d])
    ctx = ccell.cc_create_geometry([ccell.geometry_desc(cfg)])
    try:
        mats = ccell.materials(cfg)
        mats[1].rho = 0.0
        with pytest.raises(ccell.CCError):
            ccell.cc_set_materials(ctx, 0, mats)
        with pytest.raises(ccell.CCError):
            ccell.cc_set_materials(ctx, 5, ccell.materials(cfg))   # no such instance
        src = ccell.source(cfg)
        src.layer = 7
        with pytest.raises(ccell.CCError):
            ccell.cc_set_source(ctx, 0, src)
        with pytest.raises(ccell.CCError) as e:
            ccell.cc_tau_stab(ctx, 0)                               # materials not set yet
        assert e.value.status == ccell.CC_ESTATE
    finally:
        ccell.cc_destroy(ctx)


def test_default_launch_shape_per_precision():
    for precision, threads in ((ccell.FP64, 128), (ccell.MIXED, 512)):
        sol = ccell.Solver(inputs.small_case(q0=1.0), precision=precision)
        try:
            assert ccell.cc_get_launch(sol.ctx) == (4, threads, 16)
        finally:
            sol.close()


def test_mixed_only_launch_shapes():
    for precision, ok in ((ccell.FP64, False), (ccell.MIXED, True)):
        sol = ccell.Solver(inputs.small_case(q0=1.0), precision=precision)
        try:
            for shape in ((4, 512, 16), (5, 512, 16), (5, 384, 16), (5, 128, 8)):
                if ok:
                    sol.set_launch(*shape)
                    assert ccell.cc_get_launch(sol.ctx) == shape
                else:  # launch mode 5 and 512-thread blocks: mixed precision only
                    with pytest.raises(ccell.CCError):
                        sol.set_launch(*shape)
            for bad in ((0, 512, 16), (6, 128, 16), (3, 384, 16)):
                with pytest.raises(ccell.CCError):
                    sol.set_launch(*bad)
        finally:
            sol.close()


def test_launch_shape_validation_and_round_trip():
    cfg = inputs.small_case(q0=1.0)
    sol = ccell.Solver(cfg)
    try:
        for shape in ((1, 64, 4), (0, 256, 16), (1, 128, 8), (2, 256, 16), (2, 64, 4),
                      (3, 128, 16), (4, 256, 16), (4, 64, 2), (4, 384, 16)):
            sol.set_launch(*shape)
            assert ccell.cc_get_launch(sol.ctx) == shape
        for bad in ((5, 128, 16), (-1, 128, 16), (0, 96, 16), (0, 128, 1), (0, 128, 32),
                    (0, 384, 16), (2, 384, 16)):
            with pytest.raises(ccell.CCError):
                sol.set_launch(*bad)
    finally:
        sol.close()


def test_no_cpu_fallback():
    """The binding refuses host tensors: every step of the path runs on the GPU."""
    torch = pytest.importorskip("torch")
    cfg = inputs.small_case(q0=1.0)
    sol = ccell.Solver(cfg)
    try:
        T = torch.tensor(inputs.initial_field(cfg).ravel())         # host memory
        target = torch.zeros(4, dtype=torch.float64)
        for call in (lambda: sol.step(T, 2), lambda: sol.step_adi(T, 2),
                     lambda: sol.autotune(T), lambda: sol.adjoint(T, 4, 0.0, 0.0, target)):
            with pytest.raises(ValueError):
                call()
    finally:
        sol.close()


@pytest.mark.parametrize("threads,rows,blocks,precision", [
    (256, 16, 152, 0), (128, 16, 304, 1), (64, 4, 456, 1), (256, 8, 0, 0), (128, 16, 7, 0)])
def test_tile_partition_covers_every_line_once(threads, rows, blocks, precision):
    """Host logic of the step launches: the CTA tiles of a ragged batch cover
    every interior line of every instance exactly once, within the tile's
    lanes and shared memory, and n blocks take contiguous tile ranges of equal
    node shares (within one line)."""
    cfgs = inputs.batched_cases(seed=1, n=24)
    descs = [ccell.geometry_desc(c, precision) for c in cfgs]
    tiles, cta, lanes, smem = ccell.cc_query_tiles(descs, threads, rows, blocks)
    assert 0 < smem <= 226 * 1024
    for k, c in enumerate(cfgs):
        G = int(lanes[k])
        assert G in (1, 2, 4, 8, 16, 32) and -(-c["nr"] // G) <= 16
        mine = tiles[tiles[:, 0] == k]
        lines = np.concatenate([np.arange(j0, j0 + nl) for _, j0, nl in mine])
        assert np.array_equal(np.sort(lines), np.arange(1, c["nz"] - 1)), k
        assert mine[:, 2].min() >= 1 and mine[:, 2].max() <= (threads // 32) * (32 // G)
    if blocks:
        assert cta[0] == 0 and cta[-1] == len(tiles) and np.all(np.diff(cta) >= 0)
        nr = np.array([c["nr"] for c in cfgs])
        per_tile = nr[tiles[:, 0]] * tiles[:, 2]
        total = int(per_tile.sum())
        assert total == sum(c["nr"] * (c["nz"] - 2) for c in cfgs)
        share = total / blocks
        block_nodes = [int(per_tile[cta[b]:cta[b + 1]].sum()) for b in range(blocks)]
        assert max(abs(x - share) for x in block_nodes) < nr.max() + 1, (min(block_nodes), share)
        # a block's run of one instance: the fewest tiles that fit, sizes within one line
        cap = {k: (threads // 32) * (32 // int(lanes[k])) for k in range(len(cfgs))}
        for b in range(blocks):
            run = tiles[cta[b]:cta[b + 1]]
            for k in np.unique(run[:, 0]):
                nl = run[run[:, 0] == k][:, 2]
                assert nl.max() - nl.min() <= 1, (b, k, nl)
                assert len(nl) == -(-int(nl.sum()) // cap[k]), (b, k, nl)


def test_entry_points_refuse_before_any_device_work():
    """Argument errors and unsupported requests return before the library
    touches the device (the pointer below is never dereferenced)."""
    fake = 256
    cfg = inputs.small_case(q0=1.0)
    sol = ccell.Solver(cfg)
    sol_mixed = ccell.Solver(cfg, precision=ccell.MIXED)
    stepped = dict(cfg, step=dict(layers=2, z=6e-3))
    sol_stepped = ccell.Solver(stepped)
    try:
        def status(fn):
            with pytest.raises(ccell.CCError) as e:
                fn()
            return e.value.status
        assert status(lambda: ccell.cc_step_n(sol.ctx, fake, -1, 0.0, 0.0, None, None, None)) \
            == ccell.CC_EINVAL
        assert status(lambda: ccell.cc_step_n(sol.ctx, None, 3, 0.0, 0.0, None, None, None)) \
            == ccell.CC_EINVAL
        ccell.cc_step_n(sol.ctx, fake, 0, 0.0, 0.0, None, None, None)   # nothing to do
        assert status(lambda: ccell.cc_step_adi_n(sol_mixed.ctx, fake, 2, 0.0, 1e-6, None, None)) \
            == ccell.CC_EUNSUPPORTED
        assert status(lambda: ccell.cc_step_adi_n(sol_stepped.ctx, fake, 2, 0.0, 1e-6, None,
                                                  None)) == ccell.CC_EUNSUPPORTED
        args = (fake, 4, 0.0, 0.0, fake, 256, fake, fake, None, None)
        assert status(lambda: ccell.cc_adjoint(sol_mixed.ctx, *args)) == ccell.CC_EUNSUPPORTED
        assert status(lambda: ccell.cc_adjoint(sol_stepped.ctx, *args)) == ccell.CC_EUNSUPPORTED
        assert status(lambda: ccell.cc_set_dt(sol.ctx, 0, -1.0)) == ccell.CC_EINVAL
        assert status(lambda: ccell.cc_set_dt(sol.ctx, 3, 1e-6)) == ccell.CC_EINVAL
    finally:
        for s in (sol, sol_mixed, sol_stepped):
            s.close()
