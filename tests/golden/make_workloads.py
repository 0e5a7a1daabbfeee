"""Write ``workloads.json``: the geometry of the synthetic thin-film workloads.

Calls only the oracle (for kappa from the contact angle and for the
most-unstable wavelength lambda_m = 2 pi / q_m and growth rate sigma_max of
the flat film, Sec. Linear Stability Analysis).  Run from the repository
root:  ``python tests/golden/make_workloads.py``.

Workloads (square, cell-centred, no-flux walls; b = 0.1, n = 3, m = 2,
theta_c = 20 deg, M = 1/2, C = 1, h0 = 1):
  small     64^2 on 4 lambda_m, noise eps = 0.01, dt0 = 1e-3, T = 5/sigma_max
  scale2k   2048^2 on 64 lambda_m, noise eps = 0.01 (run to rupture)
  scale8k   8192^2 on 64 lambda_m, noise eps = 0.01 (200 timed steps)
  prof4k    4096^2 on 64 lambda_m (profiling captures: inputs larger than L2)
  nucl8k    8192^2 on 256 lambda_m, eps = 1e-4 + 64 Gaussian depressions
            of depth 0.3 h0 and width lambda_m / 4
  adjoint1k 1024^2 on 16 lambda_m, spinodal noise eps = 0.01: the step with
            exactly 3 Newton iterations at dt = 0.01, where 3 iterations
            bring max|v/u| to 8e-5 (10 iterations: 7e-11).  At dt =
            (2/sigma_max)/400 = 47.6 the 3-iteration map from this film
            diverges (max|v/u| = 569, a non-positive iterate).  The
            trajectory: 400 such steps (T = 4); its loss |h(T) - h_target|^2
            takes h_target from the same 400 steps of the film of seed 1242.
Step control: dt_max = 0.01/sigma_max, dt_min = 1e-9, shrink 1/2, grow 5/4
after 5 accepted steps, K = 10 Newton iterations, tol 1e-10.

Model variants (Sec. Thin Film Models), the scale8k geometry in units of each
model's own lambda_m and sigma_max, the flat heights of Sec. Validation:
  nlc8k     NLC (eq. NLC_paras: C = 0.0857, b = 0.01), h0 = 0.5
  pol8k     polymer (eq. Polymer_scales: C = 0.00581), h0 = 3.9
with dt0 * sigma_max and dt_max * sigma_max equal to scale8k's.

ensemble  256 independent films (the many-film statistics runs of Sec.
          Results): per film (numpy default_rng(1240), in this order)
          N uniform in {128, 256, 512, 1024} and the contact angle
          uniform in [10, 40] deg; power law, h0 = 1, eps = 0.01, 32
          cells per lambda_m of the film's own contact angle (so N/32
          wavelengths per side), dt0 = 1e-7/sigma_max, dt_max =
          0.01/sigma_max, 500 attempts per film.

spectrum8k  the radial Fourier analysis (App. Radial Fourier Transform) of
          an 8192^2 film at scale8k's spacing (lambda_m / 128): a ring film
          (256 cosine modes about q_m, spread 5 %, amplitude 0.05 h0, noise
          0.002 h0, seed 1241), q_cut = 5 q_m, sigma = 1, 10 points per
          interval, 400 samples.
"""
import json
import math
import os
import sys

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
import oracle as O  # noqa: E402


def main():
    b, n, m, th = 0.1, 3, 2, math.radians(20.0)
    kappa = O.kappa_from_contact_angle(th, b, n, m)
    M = O.Model(nx=1, ny=1, ds=1.0, kappa=kappa, b=b, n=n, m=m)
    qm, sm = O.lsa(M, 1.0)
    lam = 2.0 * math.pi / qm
    common = dict(model=0, b=b, n=n, m=m, theta_c=th, kappa=kappa, cap_C=1.0, h0=1.0,
                  theta=0.5, lambda_m=lam, sigma_max=sm, tol=1e-10, max_iter=10,
                  dt_min=1e-9, dt_max=0.01 / sm, dt_shrink=0.5, dt_grow=1.25,
                  grow_after=5, rupture_h=2.0 * b)
    W = {
        "small": dict(common, N=64, P=4, eps=0.01, seed=1234, dt0=1e-3, T=5.0 / sm),
        "scale2k": dict(common, N=2048, P=64, eps=0.01, seed=1235, dt0=1e-3, T=1e30),
        "scale8k": dict(common, N=8192, P=64, eps=0.01, seed=1235, dt0=1e-3, T=1e30,
                        steps=200),
        "prof4k": dict(common, N=4096, P=64, eps=0.01, seed=1237, dt0=1e-3, T=1e30),
        "nucl8k": dict(common, N=8192, P=256, eps=1e-4, seed=1236, dt0=1e-3, T=1e30,
                       holes=64, depth=0.3, width=lam / 4.0),
        "adjoint1k": dict(common, N=1024, P=16, eps=0.01, seed=1238, dt0=1e-3,
                          T=1e30, dt_fixed=0.01, fixed_iter=3, steps=400, target_seed=1242),
    }
    for w in W.values():
        w["ds"] = w["P"] * lam / w["N"]
    # model variants: NLC (model 2) and polymer (model 3)
    for name, model, C, bb, h0 in (("nlc8k", 2, 0.0857, 0.01, 0.5), ("pol8k", 3, 0.00581, 0.1, 3.9)):
        Mv = O.Model(nx=1, ny=1, ds=1.0, model=model, cap_C=C, b=bb)
        qv, sv = O.lsa(Mv, h0)
        lv = 2.0 * math.pi / qv
        W[name] = dict(common, model=model, cap_C=C, b=bb, h0=h0, lambda_m=lv, sigma_max=sv,
                       N=8192, P=64, eps=0.01, seed=1239, dt0=1e-3 * sm / sv, T=1e30,
                       dt_max=0.01 / sv, steps=40, ds=64 * lv / 8192, rupture_h=0.0)
    import numpy as np
    rng = np.random.default_rng(1240)
    films = []
    for i in range(256):
        N = int(rng.choice([128, 256, 512, 1024]))
        thc = float(rng.uniform(10.0, 40.0))
        kv = O.kappa_from_contact_angle(math.radians(thc), b, n, m)
        qv, sv = O.lsa(O.Model(nx=1, ny=1, ds=1.0, kappa=kv, b=b, n=n, m=m), 1.0)
        lv = 2.0 * math.pi / qv
        films.append(dict(N=N, theta_c_deg=thc, kappa=kv, lambda_m=lv, sigma_max=sv,
                          ds=lv / 32.0, P=N / 32.0, seed=2000 + i, dt0=1e-7 / sv, dt_max=0.01 / sv))
    W["ensemble"] = dict(common, cells_per_lambda=32, eps=0.01, attempts=500, films=films)
    W["spectrum8k"] = dict(common, N=8192, P=64, ds=64 * lam / 8192, seed=1241, eps=0.05,
                           spread=0.05, modes=256, noise=0.002, q_cut=5.0 * qm, sigma=1.0,
                           points_per_interval=10, n_eval=400, steps=50)
    out = os.path.join(os.path.dirname(__file__), "workloads.json")
    with open(out, "w") as f:
        json.dump(W, f, indent=1, sort_keys=True)
    print(out)


if __name__ == "__main__":
    main()
