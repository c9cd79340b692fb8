"""Write the stored expected values under tests/golden/ using the oracle only.

Every value here comes from the CPU oracle (`oracle/`) on seeded synthetic
inputs from `workload`; nothing is taken from the CUDA path.

    python tests/golden/make_golden.py ring8     # ring 8, (4,4), U=4: dense + Lanczos a/b
    python tests/golden/make_golden.py sq4x4     # 4x4, (8,8), U=8: matrix-free Lanczos
    python tests/golden/make_golden.py ring18 --U 4
    python tests/golden/make_golden.py ring18-bethe --U 2   # exact solution of the ring
"""
import argparse
import datetime
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle.basis import Sector  # noqa: E402
from oracle.bethe import lieb_wu_ground_energy  # noqa: E402
from oracle.kron import KronHamiltonian, lanczos_matrix_free  # noqa: E402
from oracle.lanczos import ground_energy_dense, lanczos_plain  # noqa: E402
from workload import lattice_by_name, start_vector  # noqa: E402


def _meta(cmd):
    return dict(command=cmd, host=platform.node(), machine=platform.machine(),
                cores=len(os.sched_getaffinity(0)),
                date=datetime.datetime.now(datetime.timezone.utc).isoformat(timespec="seconds"))


def _write(name, obj):
    path = os.path.join(HERE, name)
    with open(path, "w") as fh:
        json.dump(obj, fh, indent=1)
    print("wrote", path)


def ring8(args):
    ns, bonds = lattice_by_name("ring8")
    S = Sector(ns, bonds, 4, 4, 1.0, 4.0)
    H = S.explicit()
    e_dense = ground_energy_dense(H.toarray())
    v0 = start_vector(S.D, seed=1234)
    r = lanczos_plain(lambda x: H @ x, v0, 100)
    _write("ring8_n4_4_U4.json", dict(
        lattice="ring8", ns=ns, nup=4, ndn=4, t=1.0, U=4.0, seed=1234, dim=S.D,
        e0_dense=e_dense, lanczos_iters=r["iters"], lanczos_energy=r["energy"],
        alpha=list(r["a"][:30]), beta=list(r["b"][:30]), meta=_meta(" ".join(sys.argv))))


def _matrix_free(name, nup, ndn, U, tol, max_iter, fname):
    ns, bonds = lattice_by_name(name)
    t0 = time.time()
    K = KronHamiltonian(ns, bonds, nup, ndn, 1.0, U)
    v0 = np.empty(K.D)
    chunk = 1 << 26
    for s0 in range(0, K.D, chunk):                    # chunked: the generator's temporaries stay small
        n = min(chunk, K.D - s0)
        v0[s0:s0 + n] = start_vector(n, seed=1234, start=s0)

    def step(j, e, rho):
        if j % 10 == 0:
            print(f"  it {j:4d} E {e:.15f} rho {rho:.3e} ({time.time() - t0:.0f}s)", flush=True)

    r = lanczos_matrix_free(K, v0, max_iter, tol=tol, on_step=step, inplace=True)
    _write(fname, dict(
        lattice=name, ns=ns, nup=nup, ndn=ndn, t=1.0, U=U, seed=1234, dim=K.D,
        e0=r["energy"], residual=r["residual"], iters=r["iters"], tol=tol,
        alpha=list(r["a"][:30]), beta=list(r["b"][:30]),
        seconds=time.time() - t0, meta=_meta(" ".join(sys.argv))))


def ring18_bethe(U):
    ns, _ = lattice_by_name("ring18")
    e = lieb_wu_ground_energy(ns, 9, 9, 1.0, U)
    _write(f"ring18_n9_9_U{U:g}.json", dict(
        lattice="ring18", ns=ns, nup=9, ndn=9, t=1.0, U=U, dim=48620 * 48620, e0=e,
        method="Lieb-Wu Bethe-ansatz equations (oracle/bethe.py), residual <= 1e-11",
        meta=_meta(" ".join(sys.argv))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["ring8", "sq4x4", "ring18", "ring18-bethe"])
    ap.add_argument("--U", type=float, default=None)
    a = ap.parse_args()
    if a.which == "ring8":
        ring8(a)
    elif a.which == "sq4x4":
        U = 8.0 if a.U is None else a.U
        _matrix_free("sq4x4", 8, 8, U, 1e-12, 600, f"sq4x4_n8_8_U{U:g}.json")
    elif a.which == "ring18":
        U = 4.0 if a.U is None else a.U
        _matrix_free("ring18", 9, 9, U, 1e-11, 600, f"ring18_n9_9_U{U:g}.json")
    else:
        ring18_bethe(2.0 if a.U is None else a.U)


if __name__ == "__main__":
    main()
