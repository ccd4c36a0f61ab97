"""GB300 (sm_103a) adaptive GSIS kinetic hot path: a C-ABI CUDA library
(libgsis.so, declared in include/gsis.h) with a thin ctypes binding."""
from .gsis import Solver, GsisError, load, version, iterate_batch, batch_info, FIELDS, PHASES, DTYPES  # noqa: F401
