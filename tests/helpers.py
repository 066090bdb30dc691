"""Builders shared by the parity tests: the same seeded workload handed to the
oracle and to the CUDA library (each builds its own state from it)."""
import numpy as np

import oracle


def oracle_from(cap):
    s = oracle.OracleSim(cap.nx, cap.ny, tau=cap.tau, re=cap.re, rho_out=cap.rho_out, bc=cap.bc, g=cap.g,
                         seed=cap.seed)
    s.set_transfer(getattr(cap, "transfer", 0))
    for b in cap.bodies:
        i = s.add_body(b.kind, b.motion, b.xy, b.xy_ref, b.ca, b.beta, b.ka, b.density_ratio)
        if b.adhesion is not None:
            a = b.adhesion
            s.set_adhesion(i, a.n_lig, a.sigma, a.y_cr, a.y_eq, a.kf_dt, a.kr0_dt, a.xi)
    return s


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
