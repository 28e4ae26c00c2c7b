"""Pins of the oracle's ray tracer against closed forms: the mass thickness a straight ray
traverses is the sum over the volumes it crosses of density x chord length, which for the
slab and the tubes is known exactly."""
import math

import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W


def layer_areal_density(geom):
    """g/cm^2 of one layer (all its sublayers) crossed at normal incidence"""
    return sum(geom.materials[m].density * t * 0.1 for m, t in zip(geom.sub_materials, geom.sub_thickness))


def test_slab_normal_incidence():
    geom = W.slab_calorimeter()
    o = oracle.Oracle(geom)
    # a 600 mm wide view of the 400 mm wide calorimeter: the outer pixels miss it
    img = o.raytrace([0, 0, -100, 0, 0, 1, 0, 1, 0, 600, 600], 12, 12)
    xs = (np.arange(12) + 0.5) / 12 * 600 - 300
    inside = np.abs(xs) < geom.half_xy
    full = geom.n_layers * layer_areal_density(geom)
    m = np.outer(inside, inside)
    np.testing.assert_allclose(img[..., 0][m], full, rtol=1e-12)
    assert (img[..., 1][m] == geom.n_layers * len(geom.sub_materials)).all()
    assert (img[..., 0][~m] == 0).all() and (img[..., 1][~m] == 0).all()


@pytest.mark.parametrize("theta_deg", [10.0, 25.0])
def test_slab_oblique_rays_scale_as_one_over_cosine(theta_deg):
    geom = W.slab_calorimeter()
    o = oracle.Oracle(geom)
    th = math.radians(theta_deg)
    d = [math.sin(th), 0.0, math.cos(th)]
    depth = sum(geom.sub_thickness) * geom.n_layers
    # rays that enter the front face near x = -150 and leave through the back face
    x0 = -150.0 - 100.0 * math.tan(th)
    img = o.raytrace([x0, 0, -100.0, *d, 0, 1, 0, 1.0, 1.0], 1, 1)
    assert -150.0 + depth * math.tan(th) < geom.half_xy
    np.testing.assert_allclose(img[0, 0, 0], geom.n_layers * layer_areal_density(geom) / math.cos(th), rtol=1e-12)


def chord(R, b):
    return 2.0 * math.sqrt(R * R - b * b) if R > b else 0.0


@pytest.mark.parametrize("b", [0.0, 150.0, 320.0, 1000.0])
def test_barrel_rays_at_impact_parameter(b):
    geom = W.barrel_calorimeter()
    o = oracle.Oracle(geom, field_T=3.8)
    img = o.raytrace([-3000.0, b, 0.0, 1, 0, 0, 0, 0, 1, 1e-3, 1e-3], 1, 1)
    # sum over every sublayer shell [r_in, r_out] of rho x (chord(r_out) - chord(r_in))
    want = 0.0
    for r0 in geom.layer_r:
        r = r0
        for m, t in zip(geom.sub_materials, geom.sub_thickness):
            want += geom.materials[m].density * 0.1 * (chord(r + t, b) - chord(r, b))
            r += t
    np.testing.assert_allclose(img[0, 0, 0], want, rtol=1e-9)


def test_barrel_along_the_axis_and_misses():
    geom = W.barrel_calorimeter()
    o = oracle.Oracle(geom, field_T=3.8)
    r = geom.layer_r[3] + geom.sub_thickness[0] + 0.5 * geom.sub_thickness[1]  # inside the Fe of layer 3
    img = o.raytrace([r, 0.0, -5000.0, 0, 0, 1, 1, 0, 0, 1e-3, 1e-3], 1, 1)
    fe = geom.materials[geom.sub_materials[1]].density
    np.testing.assert_allclose(img[0, 0, 0], fe * 2 * geom.half_z * 0.1, rtol=1e-12)
    assert img[0, 0, 1] == 1
    miss = o.raytrace([-3000.0, 5000.0, 0.0, 1, 0, 0, 0, 0, 1, 1.0, 1.0], 2, 2)
    assert (miss == 0).all()
