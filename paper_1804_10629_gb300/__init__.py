"""GB300-native s-step enlarged Krylov subspace CG (arXiv:1804.10629).

The solver is the C-ABI library libekcg.so (include/ekcg.h, sources in csrc/); `ekcg` is
its Python binding.  Build with `python -m paper_1804_10629_gb300.build`.
"""
from . import ekcg  # noqa: F401  (binding only; the library loads on first call)
