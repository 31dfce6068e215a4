"""Seeded synthetic ensembles of protein-like models (input generation only).

This module holds no part of the cRMSD arithmetic: it only draws coordinates.
Both the CUDA path (tests, bench) and the FP64 oracle's tests take their inputs
from here, so that the two sides see bit-identical FP32 coordinates.

The paper's decoy sets (Decoys 'R' Us 1ctf and vhp_mcmd, the I-TASSER decoys,
the qcprot proteins) are not available; these ensembles stand in for them with
the same shape: N models of L C-alpha atoms each, with the same atom
correspondence in every model (eq. 1 sums over matched atom pairs).

Recipe (every draw from numpy ``Generator(PCG64(seed))``):

* native chain: a random walk with 3.8 A bonds; the interior bond angle at every
  atom is uniform in [80, 150] degrees and the torsion uniform in [-180, 180];
  the first bond lies along +x; no self-avoidance;
* model: native + i.i.d. N(0, sigma^2) on every coordinate, sigma drawn per
  model from the configuration's range, then a Haar-uniform rotation (a
  normalised 4-D Gaussian quaternion) and a translation uniform in [-50, 50]^3,
  then a cast to float32;
* model order: a seeded permutation, so that tile-level structure is not
  order-lucky.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOND = 3.8
SEED_BASE = 13024000


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def native_chain(L: int, rng: np.random.Generator) -> np.ndarray:
    """A random-walk C-alpha trace of L atoms (float64, shape [L, 3])."""
    x = np.zeros((L, 3), dtype=np.float64)
    if L == 1:
        return x
    theta = np.deg2rad(rng.uniform(80.0, 150.0, size=L))
    phi = np.deg2rad(rng.uniform(-180.0, 180.0, size=L))
    x[1] = (BOND, 0.0, 0.0)
    if L == 2:
        return x
    t = theta[1]
    x[2] = x[1] + BOND * np.array([-math.cos(t), math.sin(t), 0.0])
    for i in range(3, L):
        a, b, c = x[i - 3], x[i - 2], x[i - 1]
        bc = c - b
        bc /= np.linalg.norm(bc)
        n = np.cross(b - a, bc)
        n /= np.linalg.norm(n)
        m = np.cross(n, bc)
        t, p = theta[i - 1], phi[i]
        d = (-BOND * math.cos(t), BOND * math.sin(t) * math.cos(p), BOND * math.sin(t) * math.sin(p))
        x[i] = c + d[0] * bc + d[1] * m + d[2] * n
    return x


def haar_rotations(n: int, rng: np.random.Generator) -> np.ndarray:
    """n Haar-uniform rotation matrices, shape [n, 3, 3] (float64)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def rigid_place(models: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Apply a random rotation and a translation in [-50, 50]^3 to each model."""
    n = models.shape[0]
    R = haar_rotations(n, rng)
    t = rng.uniform(-50.0, 50.0, size=(n, 1, 3))
    return np.einsum("nij,nlj->nli", R, models) + t


@dataclass
class Ensemble:
    """A synthetic ensemble: coords[N, L, 3] float32 plus provenance."""

    coords: np.ndarray
    sigma: np.ndarray
    native_id: np.ndarray
    natives: np.ndarray
    recipe: str
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.coords.shape[0]

    @property
    def L(self) -> int:
        return self.coords.shape[1]


def _finish(models, sigma, native_id, natives, rng, recipe, per_model=None) -> Ensemble:
    """Rigid placement, seeded permutation of the model order, FP32 cast; per_model arrays
    (provenance, e.g. cluster ids) are permuted with the models."""
    placed = rigid_place(models, rng)
    perm = rng.permutation(models.shape[0])
    coords = np.ascontiguousarray(placed[perm].astype(np.float32))
    extra = {k: np.asarray(v)[perm] for k, v in (per_model or {}).items()}
    return Ensemble(coords, sigma[perm], native_id[perm], natives, recipe, extra)


def decoy_ensemble(N: int, L: int, n_natives: int, sigma_range, seed: int) -> Ensemble:
    """N models split evenly over n_natives seeded natives, sigma ~ U(sigma_range)."""
    ss = np.random.SeedSequence(seed)
    child = ss.spawn(n_natives + 1)
    natives = np.stack([native_chain(L, _rng(c)) for c in child[:n_natives]])
    rng = _rng(child[n_natives])
    native_id = np.arange(N) % n_natives
    sigma = rng.uniform(sigma_range[0], sigma_range[1], size=N)
    noise = rng.standard_normal((N, L, 3)) * sigma[:, None, None]
    models = natives[native_id] + noise
    recipe = (f"decoys: N={N} L={L} natives={n_natives} sigma~U{tuple(sigma_range)} seed={seed}")
    return _finish(models, sigma, native_id, natives, rng, recipe)


def config0(seed: int = SEED_BASE + 0) -> Ensemble:
    """Small plain-method case: 200 models x 100 atoms, one native, sigma 0.5-8 A."""
    return decoy_ensemble(200, 100, 1, (0.5, 8.0), seed)


def config1(seed: int = SEED_BASE + 1, N: int = 5000, L: int = 300) -> Ensemble:
    """Plain method at scale: 5,000 x 300 from 5 natives (1,000 each), sigma 0.5-10 A."""
    return decoy_ensemble(N, L, 5, (0.5, 10.0), seed)


def config2(seed: int = SEED_BASE + 2, N: int = 20000, L: int = 150, n_natives: int = 10,
            n_centres: int = 500) -> Ensemble:
    """Precision case: half diverse (sigma 1-8 A), half near-duplicate clusters.

    The near-duplicate half is n_centres cluster centres (native + sigma 1-8 A),
    each with N/2/n_centres members drawn around the centre with sigma 0.02-0.5 A.
    """
    ss = np.random.SeedSequence(seed)
    child = ss.spawn(n_natives + 1)
    natives = np.stack([native_chain(L, _rng(c)) for c in child[:n_natives]])
    rng = _rng(child[n_natives])
    n_div = N // 2
    n_dup = N - n_div
    per = max(1, n_dup // n_centres)
    nid_div = rng.integers(0, n_natives, size=n_div)
    sig_div = rng.uniform(1.0, 8.0, size=n_div)
    div = natives[nid_div] + rng.standard_normal((n_div, L, 3)) * sig_div[:, None, None]
    nid_c = rng.integers(0, n_natives, size=n_centres)
    sig_c = rng.uniform(1.0, 8.0, size=n_centres)
    centres = natives[nid_c] + rng.standard_normal((n_centres, L, 3)) * sig_c[:, None, None]
    cid = np.minimum(np.arange(n_dup) // per, n_centres - 1)
    sig_m = rng.uniform(0.02, 0.5, size=n_dup)
    dup = centres[cid] + rng.standard_normal((n_dup, L, 3)) * sig_m[:, None, None]
    models = np.concatenate([div, dup])
    sigma = np.concatenate([sig_div, sig_m])
    native_id = np.concatenate([nid_div, nid_c[cid]])
    recipe = (f"precision: N={N} L={L} natives={n_natives}; {n_div} diverse sigma~U(1,8); "
              f"{n_centres} centres x {per} members sigma~U(0.02,0.5) seed={seed}")
    cluster = np.concatenate([np.full(n_div, -1), cid])  # near-duplicate cluster id, -1 for diverse models
    return _finish(models, sigma, native_id, natives, rng, recipe, {"cluster": cluster})


def config3(seed: int = SEED_BASE + 3, N: int = 1024, L: int = 256, n_close: int = 10):
    """Differentiation case: 1,024 x 256, one native, sigma 0.5-8 A, plus weights.

    n_close disjoint pairs (2k, 2k+1 before the final permutation) are rebuilt so
    that model b is a rigid copy of model a with N(0, (2e-4)^2) noise, giving
    cRMSD of about 3.5e-4 A, below the 1e-3 A guard scale. Returns the ensemble
    and the condensed weights w_ab ~ U[0, 1].
    """
    ss = np.random.SeedSequence(seed)
    c_nat, c_rest = ss.spawn(2)
    native = native_chain(L, _rng(c_nat))
    rng = _rng(c_rest)
    sigma = rng.uniform(0.5, 8.0, size=N)
    models = native[None] + rng.standard_normal((N, L, 3)) * sigma[:, None, None]
    placed = rigid_place(models, rng)
    for k in range(n_close):
        a, b = 2 * k, 2 * k + 1
        ca = placed[a] - placed[a].mean(axis=0)
        Q = haar_rotations(1, rng)[0]
        t = rng.uniform(-50.0, 50.0, size=3)
        placed[b] = (ca + rng.standard_normal((L, 3)) * 2e-4) @ Q.T + t
    perm = rng.permutation(N)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(N)
    close_pairs = [tuple(sorted((int(inv[2 * k]), int(inv[2 * k + 1])))) for k in range(n_close)]
    coords = np.ascontiguousarray(placed[perm].astype(np.float32))
    P = N * (N - 1) // 2
    w = rng.uniform(0.0, 1.0, size=P).astype(np.float32)
    ens = Ensemble(coords, sigma[perm], np.zeros(N, dtype=np.int64), native[None],
                   f"differentiation: N={N} L={L} sigma~U(0.5,8), {n_close} pairs at ~3.5e-4 A seed={seed}",
                   {"close_pairs": close_pairs})
    return ens, w


def config4(seed: int = SEED_BASE + 4, N: int = 50000, L: int = 1000) -> Ensemble:
    """Large combined: 10 natives, sigma 0.1-12 A (forward 50,000 x 1,000; fwd+bwd 8,192 x 500)."""
    return decoy_ensemble(N, L, 10, (0.1, 12.0), seed)


def weights(P: int, seed: int) -> np.ndarray:
    """Condensed pair weights w_ab ~ U[0, 1] (float32) for the loss sum w_ab * cRMSD_ab."""
    return _rng(seed).uniform(0.0, 1.0, size=P).astype(np.float32)
