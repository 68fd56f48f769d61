"""Seeded synthetic inputs for the D-VQLS hot path.

This module only builds inputs (matrices, right-hand sides, angle vectors); it
holds none of the method's arithmetic, imports neither the CUDA binding nor
the oracle, and is the one module both sides take their inputs from.

Workloads (shapes and distributions of the paper's benchmarks, Sec. 2.5 and
Sec. 3; no dataset is involved anywhere):
  - tridiagonal Toeplitz systems (Sec. 2.5.1): diagonal a, off-diagonals c;
  - the n = 3 validation system: tridiag(-1, 2.5, -1) scaled by its spectral
    norm, b = |+>^3, depth 2 (9 angles);
  - the n = 10 throughput system: a ~ U(2,4), c ~ U(-1.5,-0.5) redrawn until
    a > 2|c| (so A is diagonally dominant), b = |+>^10, depth 4 (50 angles),
    top-64 terms;
  - a Hele-Shaw-type pressure system (Sec. 2.5.2): 5-point variable-
    permeability Laplacian on a 32 x 32 grid with Dirichlet faces,
    k = exp(0.3 g) for smooth Gaussian noise g, and a Gaussian bump source;
  - an uneven batch of tridiagonal / pentadiagonal Toeplitz instances of
    mixed size.
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def plus_state(n):
    """|+>^n as a complex128 vector."""
    N = 1 << n
    return np.full(N, 1.0 / np.sqrt(N), dtype=np.complex128)


def toeplitz_bands(n, diag):
    """Symmetric banded Toeplitz: diag = [a, c1, c2, ...] (main, first off, ...).

    Returns (offsets, band_values) with band_values[k][r] = A[r, r + offsets[k]]."""
    N = 1 << n
    offsets, vals = [], []
    for k, v in enumerate(diag):
        if k == 0:
            offsets.append(0)
            vals.append(np.full(N, float(v)))
        else:
            for o in (-k, k):
                row = np.full(N, float(v))
                if o > 0:
                    row[N - o:] = 0.0
                else:
                    row[: -o] = 0.0
                offsets.append(o)
                vals.append(row)
    return np.array(offsets, dtype=np.int32), np.stack(vals)


def dense_from_bands(n, offsets, band_values):
    N = 1 << n
    A = np.zeros((N, N))
    for o, row in zip(offsets, band_values):
        for r in range(N):
            c = r + int(o)
            if 0 <= c < N:
                A[r, c] = row[r]
    return A


def toeplitz_dense(n, a, c_off):
    """Tridiagonal Toeplitz with diagonal a and both off-diagonals c_off."""
    N = 1 << n
    A = np.diag(np.full(N, float(a)))
    A += np.diag(np.full(N - 1, float(c_off)), 1)
    A += np.diag(np.full(N - 1, float(c_off)), -1)
    return A


def random_angles(P, seed):
    """alpha ~ U(-pi, pi)^P from a seeded generator."""
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, P)


def validation_system():
    """n = 3: A = tridiag(-1, 2.5, -1) / ||A||_2, b = |+>^3, depth 2."""
    n, d = 3, 2
    A = toeplitz_dense(n, 2.5, -1.0)
    A = A / np.linalg.norm(A, 2)
    return {"n": n, "d": d, "A": A, "b": plus_state(n), "tau": 0.0, "L_max": 1 << (2 * n),
            "alphas": [random_angles(n * (d + 1), 1000 + i) for i in range(32)]}


def throughput_instance(seed, n=10, d=4, L_max=64):
    """n = 10 Toeplitz instance: a ~ U(2,4), c ~ U(-1.5,-0.5), redrawn while
    a <= 2|c|.  Returns the banded description, b = |+>^n and alpha."""
    rng = np.random.default_rng(seed)
    redraws = 0
    while True:
        a = rng.uniform(2.0, 4.0)
        c = rng.uniform(-1.5, -0.5)
        if a > 2.0 * abs(c):
            break
        redraws += 1
    offsets, bands = toeplitz_bands(n, [a, c])
    alpha = np.random.default_rng(10_000 + seed).uniform(-np.pi, np.pi, n * (d + 1))
    return {"n": n, "d": d, "a": a, "c": c, "redraws": redraws, "offsets": offsets,
            "bands": bands, "b": plus_state(n), "alpha": alpha, "tau": 0.01, "L_max": L_max}


def _smooth_noise(rng, shape, sigma):
    """White noise convolved with a periodic Gaussian of width sigma, standardised."""
    w = rng.normal(size=shape)
    ky = np.fft.fftfreq(shape[0])[:, None]
    kx = np.fft.fftfreq(shape[1])[None, :]
    g = np.fft.ifft2(np.fft.fft2(w) * np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2))).real
    return (g - g.mean()) / g.std()


def hele_shaw_pressure(seed, grid=32, d=6, L_max=256):
    """Variable-permeability 5-point Laplacian on a grid x grid mesh (n = 10 at 32).

    Cell p = iy*grid + ix (so the low qubits index x).  Face permeability is
    the arithmetic mean of its two cells; a Dirichlet boundary face adds the
    cell's own permeability to the diagonal.  b is a normalised Gaussian bump
    (sigma = 4 cells) at the centre."""
    rng = np.random.default_rng(seed)
    k = np.exp(0.3 * _smooth_noise(rng, (grid, grid), 3.0))
    N = grid * grid
    A = np.zeros((N, N))
    for iy in range(grid):
        for ix in range(grid):
            p = iy * grid + ix
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jy, jx = iy + dy, ix + dx
                if 0 <= jy < grid and 0 <= jx < grid:
                    kf = 0.5 * (k[iy, ix] + k[jy, jx])
                    A[p, p] += kf
                    A[p, jy * grid + jx] -= kf
                else:
                    A[p, p] += k[iy, ix]
    yy, xx = np.mgrid[0:grid, 0:grid]
    c0 = (grid - 1) / 2.0
    bump = np.exp(-((xx - c0) ** 2 + (yy - c0) ** 2) / (2.0 * 4.0 ** 2)).ravel()
    b = (bump / np.linalg.norm(bump)).astype(np.complex128)
    n = int(round(np.log2(N)))
    alpha = np.random.default_rng(20_000 + seed).uniform(-np.pi, np.pi, n * (d + 1))
    return {"n": n, "d": d, "A": A, "b": b, "alpha": alpha, "tau": 0.001, "L_max": L_max}


def uneven_batch(seed=0, count=62, big=2, sizes=(4, 6, 8, 10, 12), big_n=20, L_max=64):
    """Mixed-size Toeplitz instances: `count` with n drawn from `sizes` (half
    tridiagonal, half pentadiagonal; off-diagonals ~ U(-1.5, 4), then the main
    diagonal raised to 1.05 * sum|off| when smaller), plus `big` tridiagonal
    instances at n = big_n.  Depth d = n/2 for each; b = |+>^n."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count + big):
        if i < count:
            n = int(rng.choice(sizes))
            nb = 1 if i % 2 == 0 else 2
        else:
            n, nb = big_n, 1
        off = rng.uniform(-1.5, 4.0, nb)
        a = rng.uniform(-1.5, 4.0)
        a = max(a, 1.05 * 2.0 * float(np.sum(np.abs(off))))
        offsets, bands = toeplitz_bands(n, [a] + list(off))
        d = n // 2
        alpha = np.random.default_rng(30_000 + 97 * seed + i).uniform(-np.pi, np.pi, n * (d + 1))
        out.append({"n": n, "d": d, "offsets": offsets, "bands": bands, "b": plus_state(n),
                    "alpha": alpha, "tau": 0.01, "L_max": L_max})
    return out


def gaussian_rhs(N, count, seed):
    """`count` normalised Gaussian right-hand sides of length N."""
    B = np.random.default_rng(seed).normal(size=(count, N))
    return B / np.linalg.norm(B, axis=1, keepdims=True)
