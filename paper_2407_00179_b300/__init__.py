"""B300-native data-parallel volume rendering: per-rank brick ray-march and
sort-last compositing with an adjoint pass (arXiv 2407.00179).

Submodules: `dpv` binds the CUDA library libdpv.so (C ABI in include/dpv.h);
`inputs` makes seeded synthetic scenes; `build` compiles the library for
sm_103a.
"""
