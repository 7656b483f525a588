"""GB300-native (sm_103a) volumetric-ray-casting fluence estimator.

The compute path is libvrc (CUDA kernels behind the C ABI in include/vrc.h);
``paper_1706_07476_gb300.vrc`` is its Python binding.  Importing the package
itself loads nothing, so that build tooling can run without a built library.
"""

__version__ = "0.1.0"
