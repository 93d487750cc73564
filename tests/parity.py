"""The parity rules of the GPU tests: oracle.compare, strict (the first violation fails)."""
from oracle.compare import COEF_RTOL, MARGIN, RESID_RTOL, RESID_YTOL, ParityError  # noqa: F401
from oracle.compare import compare as _compare


def compare(*args, **kw):
    kw.setdefault("strict", True)
    return _compare(*args, **kw)
