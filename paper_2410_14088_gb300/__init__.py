"""GB300-native compressed full-state quantum circuit simulator (after BMQSim,
arXiv 2410.14088).

  * `qsim`   — Python binding of the C ABI in include/qsim.h (libqsim.so);
  * `inputs` — seeded synthetic circuits and amplitude blocks;
  * `build`  — in-tree nvcc build of libqsim.so for sm_103a.

Import the submodules explicitly; importing the package loads nothing.
"""
