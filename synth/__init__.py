"""Seeded synthetic edge-point workloads.

This package only draws inputs: binary edge images made of rasterised segments
plus salt noise, returned as int16 (x, y) point lists, and grey-level images
for the front end.  It holds none of the
Hough-transform arithmetic, so both the CPU oracle and the CUDA path can share
it without sharing any of the method.
"""
from .edges import (  # noqa: F401
    EdgeImage,
    edge_points,
    plain_128,
    plain_1024,
    plain_4096,
    batch_256,
    serving_requests,
    serving_request,
    batch_image,
    random_small,
    poisson_arrivals,
    Stream,
    ceil_log2,
    CONFIG_SEED_BASE,
)
from .gray import GrayImage, gray_256, gray_4096, gray_random  # noqa: F401
