"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This package renders star fields, sky, noise, detector defects and PSF stamps.
It holds none of the catalog method's arithmetic (no background estimation,
thresholding, labeling, centroiding, photometry or PSF fitting): both the CUDA
path and the CPU oracle consume what it writes.
"""
from .frames import (  # noqa: F401
    FrameTruth,
    frame_field,
    frame_field_device,
    frame_gradient_1k,
    frame_survey_4k,
    raw_calibrated_4k,
    moffat_stamps,
    tiny_frame,
    mixed_batch_shapes,
    wcs_pair,
)
