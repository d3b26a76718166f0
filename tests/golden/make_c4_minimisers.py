"""Write tests/golden/c4_minimisers.npz: oracle minimisers of eight requests of
the n = 5440, T = 12000 frontier sweep (GARCH sector panel, seed 3).

The sweep has 64 requests: preference vectors (1, 1, l3, l4), l3, l4 in
{0.5, 2}, times 16 return targets at the asset-mean quantiles 0.40 .. 0.85;
request q = 16 * (vector index) + (target index).  This script keeps the two
extreme targets of every vector (q = 16 v and 16 v + 15).  Three vectors
satisfy the coefficient-only convexity certificate (Cor. coefficient-only
convexity: 8 c2 c4 > 3 c3^2); (1, 1, 2, 0.5) does not, so its stored point
is the oracle's KKT point from the same start, not a certified minimiser.

Each request is solved by the oracle alone: the mean coefficient calibrated
to the target (Sec. 6) with a gap tolerance of 1e-12 max|mu|, every inner
YAND-MVSK solve (Alg. 1, PCG configuration, Table yand-core-parameters)
run to kkt_rel <= 1e-12.  The panel's bytes depend on the platform's libm
(the draws go through log/exp), so the file records their SHA-256 and the
machine that wrote it; the GPU test uses the stored points only when its own
panel has the same hash.  Run from the repository root:

    python tests/golden/make_c4_minimisers.py [--out PATH]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import panels  # noqa: E402
from oracle import mvsk_oracle as O  # noqa: E402

WORKLOAD = "c4_batch_n5440_T12000"
REQUESTS = [0, 15, 16, 31, 32, 47, 48, 63]
TOL = 1e-12
CAL_REL_TOL = 1e-12


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_minimisers.npz"))
    args = ap.parse_args()
    R, lams, tg = panels.workload(WORKLOAD)
    mu, A = O.centre(R)
    W, C, F, KKT, EVALS = [], [], [], [], []
    for q in REQUESTS:
        lam, target = lams[q // len(tg)], tg[q % len(tg)]
        c = O.scale_preferences(lam, A, "standardised")
        t0 = time.perf_counter()
        cc, x, info, ev = O.calibrate_target(A, mu, c, target, "pcg", TOL, rel_tol=CAL_REL_TOL,
                                             opts=O.Options(max_elapsed=600.0))
        dt = time.perf_counter() - t0
        W.append(x)
        C.append(cc)
        F.append(info.f)
        KKT.append(info.kkt_rel)
        EVALS.append(ev)
        print(f"q={q} lam={list(lam)} c1={cc[0]:.6e} status={info.status} kkt_rel={info.kkt_rel:.2e} "
              f"evals={ev} free={info.free_count} gap={(mu @ x - target) / np.max(np.abs(mu)):.1e} {dt:.1f}s",
              flush=True)
    np.savez_compressed(
        args.out, machine=platform.machine(), numpy=np.__version__,
        requests=np.asarray(REQUESTS), w=np.asarray(W), c=np.asarray(C), f=np.asarray(F),
        kkt_rel=np.asarray(KKT), evals=np.asarray(EVALS), tol=TOL, cal_rel_tol=CAL_REL_TOL,
        panel_sha256=hashlib.sha256(R.tobytes()).hexdigest(),
        certificate=np.asarray([O.convexity_certificate(c) for c in C]))


if __name__ == "__main__":
    main()
