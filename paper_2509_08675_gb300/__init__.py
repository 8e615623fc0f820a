"""GB300 (sm_103a) spectral-filtering generator of hyperuniform random fields
(arXiv 2509.08675): CUDA kernels behind the C ABI of include/hufield.h and a
thin Python binding (``paper_2509_08675_gb300.hufield``)."""

__all__ = ["build", "hufield"]


def build(force: bool = False):
    from . import builder as _b

    return _b.build(force=force)
