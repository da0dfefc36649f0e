"""Workload descriptions and seeded initial fields.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) in counter form: draw i of a
stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15); a uniform double
in [0, 1) is the top 53 bits times 2^-53.

Field layout: (m, ny, nx) float64, component-major, x fastest. The state
components are (v1, v2, F11, F12, F21, F22). Edge order: left, right, bottom,
top. Edge kinds: 'periodic', 'velocity', 'traction'.
"""
from dataclasses import dataclass, field

import numpy as np

__all__ = ["splitmix64_uniform", "Workload", "shear_wave_64", "clamped_specimen",
           "fourier_periodic", "specimen_batch", "adjoint_specimen", "gaussian_random_field",
           "standard_normals", "rest_state", "WORKLOADS"]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from the SplitMix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Edge:
    kind: str = "periodic"            # periodic | velocity | traction
    value: tuple = (0.0, 0.0)         # v_D or nominal traction T
    timefn: str = "const"             # const | linear_ramp | sin2_ramp | sin_pulse | ricker
    tparams: tuple = (0.0, 0.0, 0.0, 0.0)
    profile: object = None            # per-node factor along the edge, or None


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    lam: float
    mu: float
    c: float
    omega: float
    dx: float = 1.0
    steps: int = 1000
    storage: str = "f32"
    body_force: tuple = (0.0, 0.0)
    edges: list = field(default_factory=lambda: [Edge(), Edge(), Edge(), Edge()])
    seed: int = 0
    note: str = ""
    params: dict = field(default_factory=dict)  # workload-specific draws

    def fields(self):
        """(U0, u0) initial state and displacement, float64 (6|2, ny, nx)."""
        return _FIELD_BUILDERS[self.name](self)


def rest_state(nx, ny):
    U0 = np.zeros((6, ny, nx))
    U0[2] = 1.0
    U0[5] = 1.0
    return U0


def _shear_wave_fields(w: Workload):
    """v1 = 0.01 sin(2 pi (iy + 1/2) / ny) + U(-1e-4, 1e-4), v2 = U(-1e-4, 1e-4),
    F = I; the noise draws run node by node (iy, then ix), two per node (v1, v2)."""
    nx, ny = w.nx, w.ny
    U0 = rest_state(nx, ny)
    r = splitmix64_uniform(w.seed, 2 * nx * ny).reshape(ny, nx, 2)
    noise = 1e-4 * (2.0 * r - 1.0)
    iy = np.arange(ny)[:, None]
    U0[0] = 0.01 * np.sin(2.0 * np.pi * (iy + 0.5) / ny) + noise[..., 0]
    U0[1] = noise[..., 1]
    return U0, np.zeros((2, ny, nx))


def _rest_fields(w: Workload):
    return rest_state(w.nx, w.ny), np.zeros((2, w.ny, w.nx))


def _fourier_fields(w: Workload, modes=16, amp=0.05, kmax=8):
    """v = sum_m (amp / modes) p_m cos(2 pi (kx X + ky Y) / L + phi_m) with integer
    (kx, ky) in [-kmax, kmax]^2 without (0, 0), a unit polarisation p_m and a
    phase phi_m, all drawn from the seeded stream; F = I. The same wave set on a
    smaller grid gives the same field in normalised coordinates."""
    nx, ny = w.nx, w.ny
    r = splitmix64_uniform(w.seed, 8 * modes)
    U0 = rest_state(nx, ny)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    n = 2 * kmax + 1
    # cos(A + B) = cos B cos A - sin B sin A with A along x and B along y, so
    # each velocity component is a rank-2*modes product (ny x 2m) @ (2m x nx)
    Ay = np.zeros((2, ny, 2 * modes))
    Bx = np.zeros((2 * modes, nx))
    for m in range(modes):
        a = r[8 * m: 8 * m + 8]
        kx = int(a[0] * n) - kmax
        ky = int(a[1] * n) - kmax
        if kx == 0 and ky == 0:
            kx = 1
        th = 2.0 * np.pi * a[2]
        phi = 2.0 * np.pi * a[3]
        ax = 2.0 * np.pi * kx * x + phi
        by = 2.0 * np.pi * ky * y
        Bx[2 * m] = np.cos(ax)
        Bx[2 * m + 1] = np.sin(ax)
        for c, wgt in ((0, np.cos(th)), (1, np.sin(th))):
            Ay[c, :, 2 * m] = (amp / modes) * wgt * np.cos(by)
            Ay[c, :, 2 * m + 1] = -(amp / modes) * wgt * np.sin(by)
    U0[0] = Ay[0] @ Bx
    U0[1] = Ay[1] @ Bx
    return U0, np.zeros((2, ny, nx))


_FIELD_BUILDERS = {}


def shear_wave_64(n=64, storage="f64", steps=1000, seed=0):
    """64 x 64 periodic square, NH lambda = 1, mu = 0.5, c = 5, omega = 2,
    shear wave v1 = 0.01 sin(2 pi Y / 64) plus uniform noise of 1e-4 (seed 0)."""
    w = Workload("shear_wave", n, n, lam=1.0, mu=0.5, c=5.0, omega=2.0, steps=steps,
                 storage=storage, seed=seed, note="periodic square, linear S-wave")
    return w


def clamped_specimen(nx=4096, ny=2048, storage="f32", steps=20000, omega=1.95):
    """Rectangular specimen: clamped left edge (v_D = 0), traction-free top and
    bottom, right-edge nominal traction (0.3 mu g(t), 0) with
    g = sin^2(pi t / (2 T_r)) for t < T_r, T_r = 10000 dt; NH lambda = 2, mu = 1;
    body force (0, -1e-6); c = 5, F = I and v = 0 at t = 0. omega = 1.95 keeps
    the traction edges below their measured growth threshold (about 1.975)."""
    c, mu = 5.0, 1.0
    dt = 1.0 / c
    edges = [Edge("velocity"),
             Edge("traction", (0.3 * mu, 0.0), "sin2_ramp", (10000 * dt, 0, 0, 0)),
             Edge("traction"), Edge("traction")]
    return Workload("clamped_specimen", nx, ny, lam=2.0, mu=mu, c=c, omega=omega, steps=steps,
                    storage=storage, body_force=(0.0, -1e-6), edges=edges,
                    note="clamped left, traction ramp right, traction-free top/bottom")


def fourier_periodic(n=8192, storage="f32", steps=5000, seed=1):
    """Periodic square, NH lambda = 1.5, mu = 0.75, c = 5, omega = 2, random
    Fourier velocity field (16 modes, amplitude 0.05, seed 1), F = I."""
    return Workload("fourier_periodic", n, n, lam=1.5, mu=0.75, c=5.0, omega=2.0, steps=steps,
                    storage=storage, seed=seed, note="periodic square, 16-mode random velocity")


def _batch_member_fields(w: Workload):
    """v = 0.02 (cos th, sin th) sin(pi X / Lx) sin(pi Y / Ly) with X, Y the node
    coordinates (ix + 1/2, iy + 1/2) dx and Lx = nx dx, Ly = ny dx; F = I."""
    nx, ny = w.nx, w.ny
    th = w.params["theta"]
    U0 = rest_state(nx, ny)
    sx = np.sin(np.pi * (np.arange(nx) + 0.5) / nx)
    sy = np.sin(np.pi * (np.arange(ny) + 0.5) / ny)
    prof = 0.02 * sy[:, None] * sx[None, :]
    U0[0] = np.cos(th) * prof
    U0[1] = np.sin(th) * prof
    return U0, np.zeros((2, ny, nx))


def specimen_batch(n=256, seed=2, side_min=64, side_max=1024, storage="f32", steps=2000, omega=1.95,
                   aspect_max=4.0):
    """n specimens of uneven size and material. Eight draws per specimen from
    the seeded stream (specimen k uses draws 8k .. 8k+7):
      node count N log-uniform in [side_min^2, side_max^2], aspect ratio
      A = nx / ny uniform in [1, aspect_max], nx = round(sqrt(N A)), ny = round(sqrt(N / A))
      (at least 3 each); mu uniform in [0.2, 2]; lambda / mu uniform in [1, 4];
      right, bottom and top edges each clamped (velocity 0) or traction-free
      with probability 1/2; the initial velocity direction theta uniform in
      [0, 2 pi). The left edge is clamped. NH closure, c = max(5, 3 c_P) with
      c_P = sqrt(lambda + 2 mu) (rho_0 = 1), omega = 1.95, no body force.
      With c = 2 c_P some members (e.g. member 128 of the seed-2 draw, lambda /
      mu = 3.9, clamped left and top, traction-free right and bottom) grow
      without bound after about 1000 steps in the FP64 oracle; 2.5 c_P and
      3 c_P keep it bounded over 2000 steps."""
    r = splitmix64_uniform(seed, 8 * n).reshape(n, 8)
    lo, hi = 2.0 * np.log(side_min), 2.0 * np.log(side_max)
    out = []
    for k in range(n):
        a = r[k]
        N = np.exp(lo + a[0] * (hi - lo))
        A = 1.0 + (aspect_max - 1.0) * a[1]
        nx = max(3, int(round(np.sqrt(N * A))))
        ny = max(3, int(round(np.sqrt(N / A))))
        mu = 0.2 + 1.8 * a[2]
        lam = mu * (1.0 + 3.0 * a[3])
        c = max(5.0, 3.0 * np.sqrt(lam + 2.0 * mu))
        kinds = ["velocity" if a[4 + j] < 0.5 else "traction" for j in range(3)]
        edges = [Edge("velocity")] + [Edge(kd) for kd in kinds]
        out.append(Workload("batch_member", nx, ny, lam=lam, mu=mu, c=c, omega=omega, steps=steps,
                            storage=storage, edges=edges, seed=seed, params={"theta": 2.0 * np.pi * a[7]},
                            note="member %d of a specimen batch" % k))
    return out


def standard_normals(seed: int, n: int) -> np.ndarray:
    """n standard normals by the Box-Muller transform of SplitMix64 pairs."""
    u = splitmix64_uniform(seed, 2 * n).reshape(n, 2)
    return np.sqrt(-2.0 * np.log(1.0 - u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


def gaussian_random_field(nx, ny, corr, seed):
    """Zero-mean, unit-variance periodic Gaussian random field on the node
    grid with covariance exp(-r^2 / (2 corr^2)) (r in nodes): seeded white
    noise filtered by exp(-|k|^2 corr^2 / 4) in Fourier space, normalised to
    unit sample variance."""
    w = standard_normals(seed, nx * ny).reshape(ny, nx)
    kx = 2.0 * np.pi * np.fft.fftfreq(nx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    filt = np.exp(-(ky[:, None] ** 2 + kx[None, :] ** 2) * corr ** 2 / 4.0)
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    g -= g.mean()
    return g / g.std()


def _adjoint_fields(w: Workload):
    """Gaussian velocity pulse v = A (cos th, sin th) exp(-|X - X_c|^2 / (2 r^2))
    at X_c = (0.3 nx, 0.5 ny) nodes, r = nx / 32 nodes, A = 0.01; F = I."""
    nx, ny = w.nx, w.ny
    p = w.params
    X = np.arange(nx) + 0.5
    Y = np.arange(ny) + 0.5
    r2 = (X[None, :] - 0.3 * nx) ** 2 + (Y[:, None] - 0.5 * ny) ** 2
    prof = p["amp"] * np.exp(-r2 / (2.0 * p["radius"] ** 2))
    U0 = rest_state(nx, ny)
    U0[0] = np.cos(p["theta"]) * prof
    U0[1] = np.sin(p["theta"]) * prof
    return U0, np.zeros((2, ny, nx))


def adjoint_specimen(n=1024, seed=3, steps=2000, corr=None, sigma=0.3, nsens=64, record_every=20,
                     storage="f32", omega=1.95):
    """Clamped-left square specimen (traction-free right, bottom and top
    edges) with a log-normal shear-modulus field mu = exp(sigma g), g a
    Gaussian random field of correlation length corr nodes (n / 16 by
    default, 64 at n = 1024) drawn with `seed`; lambda = 2 mu; NH; a Gaussian
    velocity pulse (direction from draw 0 of stream seed + 1); c = max(5,
    3 c_P,max), c_P,max = sqrt(4 max mu). Sensors: nsens nodes on the right
    edge at rows (j + 1/2) n / nsens; records every record_every steps.
    Target displacements d = 1e-3 (2 U - 1) from stream seed + 2 (a synthetic
    observation), shaped (records, sensors, 2). The field, sensors, records
    and targets are in params."""
    corr = n / 16.0 if corr is None else corr
    mu = np.exp(sigma * gaussian_random_field(n, n, corr, seed))
    c = max(5.0, 3.0 * np.sqrt(4.0 * mu.max()))
    sens = np.array([[n - 1, int((j + 0.5) * n / nsens)] for j in range(nsens)], dtype=np.int32)
    rec = np.arange(record_every, steps + 1, record_every, dtype=np.int32)
    tgt = 1e-3 * (2.0 * splitmix64_uniform(seed + 2, len(rec) * nsens * 2) - 1.0)
    theta = 2.0 * np.pi * splitmix64_uniform(seed + 1, 1)[0]
    edges = [Edge("velocity"), Edge("traction"), Edge("traction"), Edge("traction")]
    return Workload("adjoint_specimen", n, n, lam=2.0 * float(mu.mean()), mu=float(mu.mean()), c=c, omega=omega,
                    steps=steps, storage=storage, edges=edges, seed=seed,
                    params={"mu": mu, "lam_ratio": 2.0, "sensors": sens, "records": rec,
                            "target": tgt.reshape(len(rec), nsens, 2), "theta": theta, "amp": 0.01,
                            "radius": n / 32.0},
                    note="clamped-left specimen, log-normal mu(X), velocity pulse, right-edge sensors")


_FIELD_BUILDERS["shear_wave"] = _shear_wave_fields
_FIELD_BUILDERS["adjoint_specimen"] = _adjoint_fields
_FIELD_BUILDERS["batch_member"] = _batch_member_fields
_FIELD_BUILDERS["clamped_specimen"] = _rest_fields
_FIELD_BUILDERS["fourier_periodic"] = _fourier_fields

WORKLOADS = {
    "shear_wave_64": shear_wave_64,
    "clamped_specimen": clamped_specimen,
    "fourier_periodic": fourier_periodic,
    "specimen_batch": specimen_batch,
    "adjoint_specimen": adjoint_specimen,
}
