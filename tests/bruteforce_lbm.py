"""Independent brute-force transcription of one STG-LBM time step.

Plain Python floats, one population at a time, with its own lattice tables
(generated by enumerating the velocity set rather than typed in) and no loop
fusion.  Used only to cross-check the oracle on tiny lattices.  Population
arrays are matched to the library's documented order by velocity vector.
"""
import itertools
import math

CS2 = 1.0 / 3.0


def lattice():
    vel = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2]
    w = {}
    for v in vel:
        n = sum(a * a for a in v)
        w[v] = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[n]
    return vel, w


VEL, W = lattice()


def feq(rho, u, v):
    cu = sum(v[a] * u[a] for a in range(3))
    uu = sum(u[a] * u[a] for a in range(3))
    return W[v] * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))


def Qab(v, a, b):
    return v[a] * v[b] - (CS2 if a == b else 0.0)


def rebuild(f, rho, u, unknown):
    """Regularized rebuild: unknown directions take the opposite's neq."""
    fneq = {}
    for v in VEL:
        if not unknown(v):
            fneq[v] = f[v] - feq(rho, u, v)
    for v in VEL:
        if unknown(v):
            o = tuple(-a for a in v)
            fneq[v] = fneq[o]
    Pi = [[sum(Qab(v, a, b) * fneq[v] for v in VEL) for b in range(3)] for a in range(3)]
    return {v: feq(rho, u, v) + W[v] / (2 * CS2 * CS2) * sum(Qab(v, a, b) * Pi[a][b]
                                                           for a in range(3) for b in range(3))
            for v in VEL}


def collide(f, tau0, C, F, regularized=True):
    rho = sum(f[v] for v in VEL)
    u = [(sum(f[v] * v[a] for v in VEL) + 0.5 * F[a]) / rho for a in range(3)]
    neq = {v: f[v] - feq(rho, u, v) for v in VEL}
    Pi = [[sum(v[a] * v[b] * neq[v] for v in VEL) for b in range(3)] for a in range(3)]
    a1 = [sum(v[a] * neq[v] for v in VEL) for a in range(3)]
    Qh = math.sqrt(sum(Pi[a][b] ** 2 for a in range(3) for b in range(3)))
    tau = tau0 / 2 + math.sqrt((tau0 * rho) ** 2 + 18 * math.sqrt(2) * C * Qh) / (2 * rho)
    out = {}
    for v in VEL:
        cu = sum(v[a] * u[a] for a in range(3))
        guo = (1 - 1 / (2 * tau)) * W[v] * sum(((v[a] - u[a]) / CS2 + cu * v[a] / CS2 ** 2) * F[a]
                                                for a in range(3))
        if regularized:
            reg = W[v] * sum(v[a] * a1[a] for a in range(3)) / CS2 + W[v] / (2 * CS2 ** 2) * sum(
                Qab(v, a, b) * Pi[a][b] for a in range(3) for b in range(3))
            out[v] = feq(rho, u, v) + (1 - 1 / tau) * reg + guo
        else:
            out[v] = f[v] - neq[v] / tau + guo
    return out


def step(pops, dims, order, tau0, C, F, u_bc, bc_x="stg", bc_y="walls", regularized=True):
    """One step.  pops[i][z][y][x] nested lists/arrays in ``order``; u_bc[c][z][y]."""
    nx, ny, nz = dims
    idx = {tuple(int(a) for a in v): i for i, v in enumerate(order)}
    new = [[[[0.0] * nx for _ in range(ny)] for _ in range(nz)] for _ in range(19)]

    def pull(x, y, z):
        f = {}
        for v in VEL:
            xs, ys, zs = x - v[0], y - v[1], (z - v[2]) % nz
            if bc_y == "walls" and not (0 <= ys < ny):
                o = tuple(-a for a in v)
                f[v] = float(pops[idx[o]][z][y][x])
                continue
            ys %= ny
            if bc_x == "periodic":
                xs %= nx
            elif not (0 <= xs < nx):
                f[v] = float("nan")
                continue
            f[v] = float(pops[idx[v]][zs][ys][xs])
        return f

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                f = pull(x, y, z)
                if bc_x == "stg" and x == 0:
                    ub = [float(u_bc[a][z][y]) for a in range(3)]
                    par = sum(f[v] for v in VEL if v[0] == 0)
                    leaving = sum(f[v] for v in VEL if v[0] < 0)
                    rho_bc = (par + 2 * leaving) / (1 - ub[0])
                    f = rebuild(f, rho_bc, ub, lambda v: v[0] > 0)
                elif bc_x == "stg" and x == nx - 1:
                    # zero gradient: the velocity of the neighbour x = nx-2 at this step
                    g = pull(nx - 2, y, z)
                    r = sum(g.values())
                    uo = [(sum(g[v] * v[a] for v in VEL) + 0.5 * F[a]) / r for a in range(3)]
                    f = rebuild(f, 1.0, uo, lambda v: v[0] < 0)
                out = collide(f, tau0, C, F, regularized)
                for v in VEL:
                    new[idx[v]][z][y][x] = out[v]
    return new
