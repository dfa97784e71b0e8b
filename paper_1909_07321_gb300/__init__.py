"""GB300-native outer-region R-matrix hot path (R -> K -> Omega).

The CUDA library (csrc/, C ABI declared in include/rmgb.h) is loaded by
`paper_1909_07321_gb300.rmgb`; importing this package itself loads nothing,
so the input generators in `synth` can be used without a GPU.
"""
