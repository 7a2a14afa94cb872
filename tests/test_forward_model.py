"""The forward model's occlusion test (tests/gen/synth.py) against cases
whose answer is plain geometry (CPU only).  The oracle's pins use it as the
independent brute-force reference, so it is checked here by itself: a ray
straight up from the beam is hidden by a wire exactly when the wire axis
passes within R of it, only between source and pixel, for any orientation
of the wire axis in the plane perpendicular to the ray."""
import numpy as np

from tests.gen import synth as S

R = S.WIRE_R_MM


def _hidden(source, pixel, centre, axis=(1.0, 0.0, 0.0)):
    return bool(S.hidden_by_wire(np.asarray(source, float),
                                 np.asarray(pixel, float)[None, :],
                                 np.asarray(centre, float), axis, R)[0])


def test_vertical_ray_hidden_within_one_radius():
    src, pix = (0.0, 0.0, 0.0), (0.0, 510.0, 0.0)
    for zc, want in ((0.0, True), (0.999 * R, True), (-0.999 * R, True),
                     (1.001 * R, False), (-1.001 * R, False), (0.5, False)):
        assert _hidden(src, pix, (0.0, 0.5, zc)) is want, zc
    # the distance is measured perpendicular to the axis: moving the wire
    # centre along its own axis changes nothing
    assert _hidden(src, pix, (123.0, 0.5, 0.999 * R))
    assert not _hidden(src, pix, (-7.0, 0.5, 1.001 * R))


def test_only_between_source_and_pixel():
    src, pix = (0.0, 0.0, 0.0), (0.0, 510.0, 0.0)
    assert _hidden(src, pix, (0.0, 509.9, 0.0))
    assert not _hidden(src, pix, (0.0, 510.0 + 1.001 * R, 0.0))   # beyond the pixel
    assert not _hidden(src, pix, (0.0, -1.001 * R, 0.0))          # behind the source
    assert _hidden(src, pix, (0.0, 510.0 + 0.999 * R, 0.0))       # the pixel inside the wire


def test_slanted_ray_distance():
    """Ray from the origin to (0, Y, Z): the distance from a wire along x
    through (0, y, z) is |y Z - z Y| / sqrt(Y^2 + Z^2) (inside the segment)."""
    Y, Z = 510.0, 40.0
    n = np.hypot(Y, Z)
    for y in (0.5, 3.0, 200.0):
        z_on = y * Z / Y                                          # on the ray
        for off, want in ((0.999, True), (1.001, False)):
            z = z_on + off * R * n / Y                            # distance off * R
            assert _hidden((0, 0, 0), (0.0, Y, Z), (0.0, y, z)) is want, (y, off)


def test_axis_orientation_in_the_plane():
    """A ray along y is perpendicular to any axis in the x-z plane; a wire
    through (0, 0.5, d) with axis (cos a, 0, sin a) lies |d cos a| from it."""
    src, pix = (0.0, 0.0, 0.0), (0.0, 510.0, 0.0)
    for a in (0.0, 0.3, 1.0):
        ax = (np.cos(a), 0.0, np.sin(a))
        for off, want in ((0.999, True), (1.001, False)):
            d = off * R / np.cos(a)
            assert _hidden(src, pix, (0.0, 0.5, d), ax) is want, (a, off)
