"""Accuracy report of the GPU forms against the CPU oracles (needs a CUDA device):

    python tests/accuracy_report.py

Prints, per workload and group, the largest eigenvalue, eigenvector and reconstruction errors
(definitions in tests/parity.py) of the FP32 precision form (FP32 and FP64 invariants), the FP32
plain form and the FP64 plain form, on samples the oracle finishes quickly. Not a test: the
tests assert the tolerances, this prints the measured values.
"""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from paper_1306_6291_gb300 import kdiag as K  # noqa: E402
from parity import D_rows, definition_errors, planes_to_rows  # noqa: E402


def errs(A, lam, D):
    e = definition_errors(planes_to_rows(A), planes_to_rows(lam), D_rows(D))
    return {k: float(np.max(np.abs(v - (1 if k == "det" else 0)))) for k, v in e.items()}


def main():
    dev = "cuda:0"
    report = {}
    A, grp = W.sym3_precision(1 << 18, seed=0, device=dev)
    g = grp.cpu().numpy()
    forms = {"fp32_precision": K.make_opts(form=K.KD_FORM_MIXED),
             "fp32_precision_inv64": K.make_opts(form=K.KD_FORM_MIXED, invariants_f64=True),
             "fp32_plain": K.make_opts(form=K.KD_FORM_PLAIN)}
    for fname, o in forms.items():
        lam, D, _, _ = K.eig3(A, o)
        for k, gname in enumerate(W.GROUPS):
            idx = torch.as_tensor(np.nonzero(g == k)[0], device=dev)
            report[f"precision/{gname}/{fname}"] = errs(A[:, idx], lam[:, idx], D[:, idx])
    for fname, X in (("fp64_plain", W.sym3_uniform(65536, seed=0, device=dev)),
                     ("fp32_precision", W.sym3_uniform(65536, seed=0, device=dev).float())):
        lam, D, _, _ = K.eig3(X)
        report[f"uniform_65536/{fname}"] = errs(X, lam, D)
    X = W.sym3_normal(1 << 18, seed=3, device=dev)
    lam, D, _, _ = K.eig3(X)
    report["normal/fp32_precision"] = errs(X, lam, D)
    for k, v in report.items():
        print(f"{k:45s} lam {v['lam']:.1e}  ev*gap {v['ev']:.1e}  rec {v['rec']:.1e}  orth {v['orth']:.1e}")
    print(json.dumps(report))


if __name__ == "__main__":
    main()
