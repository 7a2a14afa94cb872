"""The oracle reproduces the stored fixture of the Sec. III-B example shape."""
import numpy as np

from oracle import oracle as O
from tests.golden.make_golden import odd_case, read_odd


def test_odd_example_shape_golden():
    images, edges, expect = read_odd()
    sc, e2 = odd_case()
    assert np.array_equal(edges, e2)
    got = O.reconstruct(sc.geom, sc.wires, images, edges)
    scale = np.abs(np.diff(images.astype(np.int64), axis=0)).sum(0)
    assert np.all(np.abs(got - expect) <= 1e-12 * np.maximum(scale, 1))
    # the stored input is what the seeded generator makes today
    assert np.array_equal(images, sc.images)
