"""GB300-native hot path of the hopping-parameter-expanded two-flavour Wilson
HMC (Hasenbusch, arXiv:1805.03560).

The compute lives in `libhmc.so` (hand-written sm_103a CUDA behind a C ABI);
`paper_1805_03560_gb300.hmc` is the thin ctypes binding.  Importing this
package loads nothing; the binding loads the library on first use and fails
loudly when it is missing.
"""
