"""The illuminated field of view over which the GPU parity tests bound the per-pixel object error."""
import numpy as np

# The scanned field of view of the per-pixel bound: object pixels whose illumination by the scan's
# starting probe, D(r) = sum_n sum_k |P0_k(r - r_n)|^2, is at least DELTA_FOV of its maximum (the
# floor delta_O max D_O of the step's denominator). Outside it the step is set by that floor rather
# than by the data: FP32 rounding of the FFTs (absolute, about 1e-7 of the field's norm) reaches
# those pixels amplified up to 1 / delta_O. The FP64 oracle run with single-precision FFTs deviates
# from itself by up to 2.7e-3 of max |O| outside on a sparse M = 256 pc-DM scan, 2.4e-5 inside.
DELTA_FOV = 1e-3


def fov_mask(positions, P, shape, M, frac=DELTA_FOV):
    P2 = np.sum(np.abs(np.asarray(P)) ** 2, axis=0)
    D = np.zeros(shape)
    for y, x in np.asarray(positions):
        D[y:y + M, x:x + M] += P2
    return D >= frac * D.max()


def probe_support(P0, frac=DELTA_FOV):
    """Probe pixels where the starting probe carries at least `frac` of its peak intensity,
    sum_k |P0_k|^2 >= frac max; outside, the probe is zero by design and its update is the same
    amplified rounding (the FP64 oracle with single-precision FFTs: 3.3e-4 of max |P| outside on the
    sparse M = 256 pc-DM scan, 7.6e-6 inside)."""
    S = np.sum(np.abs(np.asarray(P0)) ** 2, axis=0)
    return S >= frac * S.max()
