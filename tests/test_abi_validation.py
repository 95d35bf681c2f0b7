"""Argument validation of fv_create_blocks, host logic that runs before any
CUDA call (so it is tested without a GPU): every malformed block, connection
or configuration is refused with FV_ERR_INVALID_ARG and a message naming the
problem, never a CUDA error or a crash."""
import pytest

import cases
from cases.core import default_params


@pytest.fixture(scope="module")
def fv():
    import paper_2012_02925_gb300 as fv
    from paper_2012_02925_gb300 import build
    build.build()
    return fv


def _refused(fv, blocks, conns, dim, params, precision="fp64", text=""):
    with pytest.raises(fv.FvError) as e:
        fv.Solver(blocks, conns, dim, params, precision)
    assert e.value.code == fv.FV_ERR_INVALID_ARG, str(e.value)
    assert text in str(e.value), str(e.value)


def _cart(ni, nj, nk):
    return cases.BlockDesc(ni, nj, nk, None, (0.0, 0.0, 0.0), (0.1, 0.1, 0.1))


PARAMS = default_params()


def test_no_blocks(fv):
    _refused(fv, [], [], 3, PARAMS, text="no blocks")


@pytest.mark.parametrize("dims", [(0, 4, 4), (4, 0, 4), (4, 4, 0), (40000, 4, 4)])
def test_block_extents(fv, dims):
    _refused(fv, [_cart(*dims)], [], 3, PARAMS, text="extents out of range")


def test_2d_needs_one_plane(fv):
    _refused(fv, [_cart(8, 8, 2)], [], 2, PARAMS, text="nk == 1")


def test_cartesian_spacing_positive(fv):
    b = cases.BlockDesc(4, 4, 4, None, (0.0, 0.0, 0.0), (0.1, 0.0, 0.1))
    _refused(fv, [b], [], 3, PARAMS, text="spacing")


@pytest.mark.parametrize("change,text", [
    (dict(alpha=(1.0,)), "n_stages"),
    (dict(limiter=3), "limiter"),
    (dict(flux=5), "flux"),
    (dict(gamma=1.0), "gamma"),
    (dict(visc=2, mu=0.1), "visc"),
    (dict(visc=1, mu=-1.0), "viscous parameters"),
    (dict(visc=1, mu=0.1, prandtl=0.0), "viscous parameters"),
    (dict(visc=1, mu=0.1, sutherland=1, t_ref=0.0), "viscous parameters"),
])
def test_configuration(fv, change, text):
    p = dict(PARAMS)
    p.update(change)
    _refused(fv, [_cart(4, 4, 4)], [], 3, p, text=text)


def test_unknown_precision(fv):
    _refused(fv, [_cart(4, 4, 4)], [], 3, PARAMS, precision=7, text="precision")


def test_dim(fv):
    _refused(fv, [_cart(4, 4, 1)], [], 1, PARAMS, text="dim")


@pytest.mark.parametrize("conn,text", [
    (cases.Connection(2, 1, (0, 0), (4, 4), 0, 0, (0, 0), (1, 2)), "block index"),
    (cases.Connection(0, 6, (0, 0), (4, 4), 0, 0, (0, 0), (1, 2)), "face out of range"),
    (cases.Connection(0, 1, (0, 0), (5, 4), 0, 0, (0, 0), (1, 2)), "dst patch outside"),
    (cases.Connection(0, 1, (0, 0), (4, 4), 0, 0, (0, 0), (1, 1)), "signed permutation"),
    (cases.Connection(0, 1, (0, 0), (4, 4), 0, 0, (1, 0), (1, 2)), "src patch outside"),
])
def test_connection(fv, conn, text):
    _refused(fv, [_cart(4, 4, 4)], [conn], 3, PARAMS, text=text)


def test_src_thinner_than_the_ghost_depth(fv):
    conn = cases.Connection(0, 1, (0, 0), (4, 4), 1, 0, (0, 0), (1, 2))
    _refused(fv, [_cart(4, 4, 4), _cart(1, 4, 4)], [conn], 3, PARAMS, text="thinner")


def test_ghosts_filled_twice(fv):
    c = cases.Connection(0, 1, (0, 0), (4, 4), 0, 0, (0, 0), (1, 2))
    _refused(fv, [_cart(4, 4, 4)], [c, c], 3, PARAMS, text="already filled")


def test_k_faces_in_2d(fv):
    conn = cases.Connection(0, 4, (0, 0), (4, 4), 0, 5, (0, 0), (1, 2))
    _refused(fv, [_cart(4, 4, 1)], [conn], 2, PARAMS, text="2D")
