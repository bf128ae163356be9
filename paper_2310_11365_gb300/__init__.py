"""GB300-native MC-moments micro-macro Parareal (arXiv 2310.11365).

The hot path (Euler-Maruyama fine propagator with per-step mean field,
restriction, matching, coarse moment ODE and the Parareal iterator) runs in
hand-written CUDA kernels for sm_103a behind the C-ABI library libmmp.so;
`mmp` is its thin ctypes binding.  Importing this package loads nothing;
`paper_2310_11365_gb300.mmp` loads the library on first use.
"""
