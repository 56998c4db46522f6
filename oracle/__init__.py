"""CPU oracle for the SFT / ASFT Morlet transform (Yamashita & Wakahara, arXiv:2110.11866).

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` /
`--impl reference` legs of `bench.py` may import or run anything in this package. The CUDA
library never calls it and shares no code, header, table or constant generator with it.

Contents
- `morlet.py`  plain FP64 numpy: the least-squares fits (Sec. II-A, Sec. III-A), the effective
  kernels the methods reach, direct truncated convolutions (eqs. xG-xGDD, the Morlet transform),
  the ASFT shift identity (Sec. II-E), the adjoint, relative RMSE (Table I) and a CPU restatement
  of the doubling sliding sum (Algorithm 1) used as an independent check.
- `sft_dd.c` / `sft_dd.py`  the kernel-integral algorithm of Sec. II-B (prefix sum of the
  modulated input, difference across the window, demodulation, combine) and the attenuated
  recursion of Sec. II-D, both in double-double arithmetic; this is also the timed CPU baseline.

Parity status of every function is stated in its docstring ("pinned by ..."); each pin is a test
under tests/ marked `not gpu`.
"""
