"""Point orderings of ibmi_order_points (host code of the library, no GPU).

Each ordering is checked against the property that defines it: x-sort is a
stable argsort of the first coordinate; red-black takes the even then the odd
positions (Section 5.7); a Hilbert order visits the cells of a regular grid
so that consecutive cells are neighbours (the curve is continuous), in 2-D and
3-D; a k-d order splits every range at the median of its widest coordinate.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def ibmi():
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as m
    return m


def test_xsort_is_a_stable_argsort(ibmi):
    rng = np.random.default_rng(0)
    pts = rng.random((500, 2))
    pts[::7, 0] = 0.25                      # ties keep their order
    perm = ibmi.ibmi_order_points(pts, ibmi.IBMI_ORDER_XSORT)
    np.testing.assert_array_equal(perm, np.argsort(pts[:, 0], kind="stable"))


def test_identity_and_red_black(ibmi):
    pts = np.random.default_rng(1).random((11, 3))
    np.testing.assert_array_equal(ibmi.ibmi_order_points(pts, ibmi.IBMI_ORDER_IDENTITY), np.arange(11))
    np.testing.assert_array_equal(ibmi.ibmi_order_points(pts, ibmi.IBMI_ORDER_REDBLACK),
                                  [0, 2, 4, 6, 8, 10, 1, 3, 5, 7, 9])


@pytest.mark.parametrize("dim,g", [(2, 16), (3, 8)])
def test_hilbert_order_walks_grid_neighbours(ibmi, dim, g):
    """Cell centres of a g^dim grid (plus the two corners fixing the bounding
    box), shuffled: in Hilbert order every step moves to an adjacent cell and
    every cell is visited once."""
    axes = np.meshgrid(*[np.arange(g)] * dim, indexing="ij")
    cells = np.stack([a.ravel() for a in axes], 1)
    rng = np.random.default_rng(2)
    cells = cells[rng.permutation(len(cells))]
    pts = np.vstack([(cells + 0.5) / g, np.zeros((1, dim)), np.ones((1, dim))])
    perm = ibmi.ibmi_order_points(pts, ibmi.IBMI_ORDER_HILBERT)
    walk = [cells[i] for i in perm if i < len(cells)]
    steps = np.abs(np.diff(np.array(walk), axis=0)).sum(1)
    assert len(walk) == g ** dim and np.all(steps == 1)


def test_kd_order_splits_at_the_median_of_the_widest_axis(ibmi):
    rng = np.random.default_rng(3)
    pts = rng.random((257, 3)) * np.array([1.0, 3.0, 0.5])
    perm = ibmi.ibmi_order_points(pts, ibmi.IBMI_ORDER_KD)
    assert sorted(perm.tolist()) == list(range(257))

    def check(idx):
        if len(idx) <= 1:
            return
        sub = pts[idx]
        ax = int(np.argmax(sub.max(0) - sub.min(0)))
        mid = len(idx) // 2
        left, right = idx[:mid], idx[mid:]
        assert pts[left, ax].max() <= pts[right, ax].min()
        check(left)
        check(right)

    check(perm)


def test_rejects_bad_input(ibmi):
    pts = np.random.default_rng(4).random((10, 2))
    with pytest.raises(ibmi.IbmiError):
        ibmi.ibmi_order_points(pts, 9)
    pts[3, 0] = np.nan
    with pytest.raises(ibmi.IbmiError):
        ibmi.ibmi_order_points(pts, ibmi.IBMI_ORDER_XSORT)
