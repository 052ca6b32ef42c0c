"""GB300-native ANCKA hot path: KNN augmentation graph build and the
random-walk orthogonal iteration, behind the C ABI in ``include/ancka.h``.

The CUDA library is loaded lazily by :mod:`paper_2408_05459_gb300.ancka`;
importing the package itself loads nothing.
"""
__all__ = ["ancka", "synth"]
