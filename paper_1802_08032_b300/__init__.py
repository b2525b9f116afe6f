"""B300-native exact quantum-circuit simulator (state vectors and density
matrices) after QuEST (arXiv 1802.08032).

`paper_1802_08032_b300.qsim` is the Python binding of the C-ABI library
`libqsim.so`; `paper_1802_08032_b300.circuits` generates seeded workloads.
Importing the package itself loads nothing.
"""
