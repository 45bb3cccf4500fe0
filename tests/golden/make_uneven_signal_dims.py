"""Write uneven96_signal_dims.txt: the signal dimension k = Q|Lambda| - R of every slice of the
96-slice uneven workload, from the FP64 oracle alone (explicit calibration matrix C with the
masking neglected, FP64 SVD, sigma_n < 0.05 sigma_1 is null; Sec. III-A and the threshold
footnote of Sec. III-B), together with the margins of the split: the ratios
sigma_k^2 / theta and sigma_{k+1}^2 / theta with theta = 0.05^2 sigma_1^2.

Run from the repository root:  python tests/golden/make_uneven_signal_dims.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pisco_oracle as O  # noqa: E402
from paper_2302_13431_gb300.phantoms import make_case, uneven_slice_specs  # noqa: E402


def main():
    specs = uneven_slice_specs(96)
    lam = O.kernel_support((3, 3), "ellipsoid")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "uneven96_signal_dims.txt")
    lines = ["# index Q grid calib k sigma_k^2/theta sigma_{k+1}^2/theta "
             "(uneven_slice_specs(96), ellipse radius 3, thr 0.05, rows=full)"]
    for i, sp in enumerate(specs):
        case = make_case(sp["grid"], sp["num_coils"], sp["calib_shape"], seed=sp["data_seed"])
        C = O.calibration_matrix(case.calib, lam, rows="full")
        _, U_sig, sig = O.nullspace_svd(C, 0.05)
        k = U_sig.shape[1]
        theta = (0.05 * sig[0]) ** 2
        lo = sig[k] ** 2 / theta if k < sig.size else 0.0
        lines.append(f"{i} {sp['num_coils']} {sp['grid'][0]} {sp['calib_shape'][0]} {k} "
                     f"{sig[k - 1] ** 2 / theta:.6f} {lo:.6f}")
        print(lines[-1], flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
