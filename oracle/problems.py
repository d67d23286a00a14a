"""Analytic flow data (oracle; test infrastructure).

Each problem gives the body force f, the Dirichlet data g on the whole boundary and the
initial velocity v0, written out by hand (no symbolic algebra at run time):

  TG2D   Taylor-Green vortex, an exact Navier-Stokes solution, so f = 0 and g = v.
  MMS2D  the manufactured solution of the paper's convergence test (Sec. 5.1, Eq. conv-test),
         read with a minus sign on the second velocity component so that div v = 0;
         f = dv/dt + (v.grad)v - nu Lap v + grad p, g = 0, v0 = 0.
  TG3D   Taylor-Green initial field, g = v0 (tangential, time independent), f = 0.
  MMS3D  v = sin t sin(pi z) (pi sin^2(pi x) sin(2 pi y), -pi sin(2 pi x) sin^2(pi y), 0),
         p = sin t prod_j sin(pi x_j) cos(pi x_j); f analytic, g = 0.
  CAV3D  lid-driven cavity (Sec. 5.2): f = 0, v0 = 0, no-slip on the walls, and on the lid z = 1
         the velocity (sin(pi t / 4), 0, 0); the paper gives the scalar profile, read here as the
         speed of a lid sliding along x.  g is only ever evaluated at face quadrature points,
         which lie inside their faces, so z = 1 singles out the lid's points.
"""
import numpy as np

PI = np.pi


class Problem:
    name = ""
    has_exact = False

    def __init__(self, nu):
        self.nu = nu

    def f(self, x, t):
        return np.zeros_like(x)

    def g(self, x, t):
        return np.zeros_like(x)

    def v0(self, x):
        return self.g(x, 0.0)


class TG2D(Problem):
    name = "TG2D"
    has_exact = True

    def v(self, x, t):
        F = np.exp(-2.0 * PI * PI * self.nu * t)
        X, Y = x[..., 0], x[..., 1]
        return F * np.stack([np.sin(PI * X) * np.cos(PI * Y), -np.cos(PI * X) * np.sin(PI * Y)], -1)

    def p(self, x, t):
        X, Y = x[..., 0], x[..., 1]
        return 0.25 * (np.cos(2 * PI * X) + np.cos(2 * PI * Y)) * np.exp(-4.0 * PI * PI * self.nu * t)

    def g(self, x, t):
        return self.v(x, t)

    def v0(self, x):
        return self.v(x, 0.0)


class MMS2D(Problem):
    name = "MMS2D"
    has_exact = True

    def _parts(self, x):
        X, Y = x[..., 0], x[..., 1]
        sx, cx, sy, cy = np.sin(PI * X), np.cos(PI * X), np.sin(PI * Y), np.cos(PI * Y)
        v = np.stack([sx * sx * sy * cy, -sx * cx * sy * sy], -1)
        grad = np.zeros(x.shape[:-1] + (2, 2))
        grad[..., 0, 0] = 2 * PI * sx * cx * sy * cy
        grad[..., 0, 1] = PI * sx * sx * np.cos(2 * PI * Y)
        grad[..., 1, 0] = -PI * np.cos(2 * PI * X) * sy * sy
        grad[..., 1, 1] = -2 * PI * sx * cx * sy * cy
        lap = np.stack([
            2 * PI * PI * np.cos(2 * PI * X) * sy * cy - 4 * PI * PI * sx * sx * sy * cy,
            2 * PI * PI * np.sin(2 * PI * X) * sy * sy - 2 * PI * PI * sx * cx * np.cos(2 * PI * Y)], -1)
        gp = np.stack([0.5 * PI * np.cos(2 * PI * X) * np.sin(2 * PI * Y),
                       0.5 * PI * np.sin(2 * PI * X) * np.cos(2 * PI * Y)], -1)
        return v, grad, lap, gp

    def v(self, x, t):
        return np.sin(t) * self._parts(x)[0]

    def p(self, x, t):
        X, Y = x[..., 0], x[..., 1]
        return np.sin(t) * np.sin(PI * X) * np.cos(PI * X) * np.sin(PI * Y) * np.cos(PI * Y)

    def f(self, x, t):
        v, grad, lap, gp = self._parts(x)
        s, c = np.sin(t), np.cos(t)
        conv = np.einsum("...il,...l->...i", grad, v) * s * s
        return c * v + conv - self.nu * s * lap + s * gp


class TG3D(Problem):
    name = "TG3D"

    def g(self, x, t):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([np.sin(PI * X) * np.cos(PI * Y) * np.cos(PI * Z),
                         -np.cos(PI * X) * np.sin(PI * Y) * np.cos(PI * Z),
                         np.zeros_like(X)], -1)


class MMS3D(Problem):
    name = "MMS3D"
    has_exact = True

    def _parts(self, x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        sx, sy = np.sin(PI * X), np.sin(PI * Y)
        s2x, s2y, c2x, c2y = np.sin(2 * PI * X), np.sin(2 * PI * Y), np.cos(2 * PI * X), np.cos(2 * PI * Y)
        zz, dz = np.sin(PI * Z), PI * np.cos(PI * Z)
        a = PI * sx * sx * s2y
        b = -PI * s2x * sy * sy
        ax, ay = PI * PI * s2x * s2y, 2 * PI * PI * sx * sx * c2y
        bx, by = -2 * PI * PI * c2x * sy * sy, -PI * PI * s2x * s2y
        lap_a = 2 * PI ** 3 * c2x * s2y - 4 * PI ** 3 * sx * sx * s2y
        lap_b = 4 * PI ** 3 * s2x * sy * sy - 2 * PI ** 3 * s2x * c2y
        zero = np.zeros_like(X)
        v = np.stack([zz * a, zz * b, zero], -1)
        grad = np.zeros(x.shape[:-1] + (3, 3))
        grad[..., 0, :] = np.stack([zz * ax, zz * ay, dz * a], -1)
        grad[..., 1, :] = np.stack([zz * bx, zz * by, dz * b], -1)
        lap = np.stack([zz * lap_a - PI * PI * zz * a, zz * lap_b - PI * PI * zz * b, zero], -1)
        gp = 0.25 * PI * np.stack([c2x * s2y * np.sin(2 * PI * Z),
                                   s2x * c2y * np.sin(2 * PI * Z),
                                   s2x * s2y * np.cos(2 * PI * Z)], -1)
        return v, grad, lap, gp

    def v(self, x, t):
        return np.sin(t) * self._parts(x)[0]

    def p(self, x, t):
        return np.sin(t) * np.prod(np.sin(PI * x) * np.cos(PI * x), axis=-1)

    def f(self, x, t):
        v, grad, lap, gp = self._parts(x)
        s, c = np.sin(t), np.cos(t)
        conv = np.einsum("...il,...l->...i", grad, v) * s * s
        return c * v + conv - self.nu * s * lap + s * gp


class CAV3D(Problem):
    name = "CAV3D"

    def g(self, x, t):
        out = np.zeros_like(x)
        out[..., 0] = np.where(x[..., 2] > 1.0 - 1e-9, np.sin(0.25 * PI * t), 0.0)
        return out

    def v0(self, x):
        return np.zeros_like(x)


PROBLEMS = {"TG2D": TG2D, "MMS2D": MMS2D, "TG3D": TG3D, "MMS3D": MMS3D, "CAV3D": CAV3D}


def make(name, nu):
    return PROBLEMS[name](nu)
