"""GB300 (sm_103a) HPS skeleton solver: CUDA kernels behind a C ABI (libhps.so).

`paper_2511_00735_gb300.hps` is the ctypes binding of the C ABI; importing this
package does not load the library (so that the seeded input module
`paper_2511_00735_gb300.inputs` can be used on machines without a GPU).
"""
