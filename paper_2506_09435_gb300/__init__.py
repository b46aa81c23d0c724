"""GB300-native FNPF-SEM hot path (arXiv 2506.09435): Laplace solve for the
velocity potential on a free-surface-following extruded GLL spectral-element
mesh, vertical-velocity recovery, Zakharov right-hand side and ERK4, as
hand-written CUDA for sm_103a behind a C ABI (``include/fnpf.h``).

Import ``paper_2506_09435_gb300.fnpf`` for the binding; importing the package
itself loads nothing.
"""
