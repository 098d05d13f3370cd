"""Seeded synthetic inputs: iTPS site tensors, initial environments, operators.

This module produces the arrays that both the CUDA path and the CPU oracle
consume.  It holds none of the CTMRG arithmetic (no contraction, projector,
SVD or measurement); it only draws random numbers and writes down the local
operators of the models the method is run on.

Conventions
-----------
* Unit cell Lx x Ly (2 x 2 here), site index i = x + Lx*y, y pointing up
  (r = (0, 1) is the top neighbour, section 4 "correlation" definition).
* Site tensor A[s, l, u, r, d] in C order: physical index first, then the
  virtual legs left, top, right, bottom (leg order evidenced by the kagome
  example's ``virtual_dim`` lists, Appendix A).
* Environment of a site, clockwise from the top-left corner:
  C1[c_T4, c_T1], T1[c_C1, k, k', c_C2], C2[c_T1, c_T2], T2[c_C2, k, k', c_C3],
  C3[c_T2, c_T3], T3[c_C3, k, k', c_C4], C4[c_T3, c_T4], T4[c_C4, k, k', c_C1].
  In T_n, k joins the ket tensor A and k' the bra tensor A*.
* Operators are real row-major matrices O[after, before]; two-site operators
  act on the combined index (s_i * d_j + s_j), source site first (Sec. 5.2,
  the ``elements`` format).
"""
from __future__ import annotations

import numpy as np

ENV_NAMES = ("C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4")


# --------------------------------------------------------------------------
# site tensors
# --------------------------------------------------------------------------
def site_index(x: int, y: int, Lx: int = 2, Ly: int = 2) -> int:
    return (x % Lx) + Lx * (y % Ly)


def product_state_tensors(phis, D: int, noise: float, seed: int,
                          Lx: int = 2, Ly: int = 2, normalise: bool = True):
    """Product state embedded in virtual index 0 plus Gaussian noise.

    ``phis[i]`` is the local state of site i.  All noise comes from one
    ``numpy.random.default_rng(seed)`` stream, sites in index order, each
    tensor filled in C order.  With ``normalise`` each tensor is divided by
    its largest absolute element.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(Lx * Ly):
        phi = np.asarray(phis[i], dtype=np.float64)
        d = phi.shape[0]
        A = np.zeros((d, D, D, D, D))
        A[:, 0, 0, 0, 0] = phi
        A = A + noise * rng.standard_normal(A.shape)
        if normalise:
            A = A / np.max(np.abs(A))
        out.append(np.ascontiguousarray(A))
    return out


def neel_tensors(d: int, D: int, noise: float, seed: int, Lx: int = 2, Ly: int = 2):
    """Neel state (up on (x+y) even, down on odd) + noise, max|A| = 1."""
    phis = []
    for i in range(Lx * Ly):
        x, y = i % Lx, i // Lx
        phi = np.zeros(d)
        phi[0 if (x + y) % 2 == 0 else d - 1] = 1.0
        phis.append(phi)
    return product_state_tensors(phis, D, noise, seed, Lx, Ly)


def x_polarised_tensors(d: int, D: int, noise: float, seed: int, Lx: int = 2, Ly: int = 2):
    """Ferromagnetic state polarised along +x for spin S=(d-1)/2, + noise."""
    Sx = spin_ops(d)["Sx"]
    w, v = np.linalg.eigh(Sx)
    phi = v[:, np.argmax(w)]
    phi = phi * np.sign(phi[np.argmax(np.abs(phi))])
    return product_state_tensors([phi] * (Lx * Ly), D, noise, seed, Lx, Ly)


def uniform_boson_tensors(nmax: int, D: int, noise: float, seed: int, Lx: int = 2, Ly: int = 2):
    """Soft-core boson product state (1,...,1)/sqrt(nmax+1) + noise."""
    phi = np.ones(nmax + 1) / np.sqrt(nmax + 1)
    return product_state_tensors([phi] * (Lx * Ly), D, noise, seed, Lx, Ly)


def ising_peps_tensor(beta: float):
    """Tensor whose double layer is the 2D classical Ising network at K=beta.

    B = [[e^{b/2}, e^{-b/2}], [e^{-b/2}, e^{b/2}]] = W W with W symmetric
    positive definite; A[s,l,u,r,d] = W[s,l] W[s,u] W[s,r] W[s,d].  Each bond
    then carries B from the ket and B from the bra, B*B = e^{K s s'} elementwise,
    so <psi|psi> is the Ising partition function.  s = 0 <-> sigma = +1.
    """
    B = np.array([[np.exp(beta / 2), np.exp(-beta / 2)],
                  [np.exp(-beta / 2), np.exp(beta / 2)]])
    w, v = np.linalg.eigh(B)
    W = (v * np.sqrt(w)) @ v.T
    A = np.einsum("sl,su,sr,sd->slurd", W, W, W, W)
    return np.ascontiguousarray(A)


def gauged_ising_tensors(beta: float, seed: int, strength: float = 0.5):
    """The Ising PEPS tensor on all four sites of the 2x2 cell, with an
    independent random invertible matrix G = 1 + strength N(0,1) (seed) on
    each of the 8 bonds: the source site's leg toward the bond gets G, the
    target site's leg G^-1 (bonds in SQUARE_2X2_BONDS order; horizontal
    bonds join r of the source to l of the target, vertical ones u of the
    source to d of the target).  Contracting any bond gives back G G^-1 = 1
    in ket and bra alike, so the norm network -- and every observable and
    the free energy -- is the Ising model's at K = beta, while the four site
    tensors all differ."""
    rng = np.random.default_rng(seed)
    A = ising_peps_tensor(beta)
    As = [A.copy() for _ in range(4)]
    for (i, dx, dy) in SQUARE_2X2_BONDS:
        x, y = i % 2, i // 2
        j = site_index(x + dx, y + dy)
        G = np.eye(2) + strength * rng.standard_normal((2, 2))
        Gi = np.linalg.inv(G)
        if dx == 1:
            As[i] = np.einsum("slurd,rk->slukd", As[i], G)
            As[j] = np.einsum("kl,slurd->skurd", Gi, As[j])
        else:
            As[i] = np.einsum("slurd,uk->slkrd", As[i], G)
            As[j] = np.einsum("kd,slurd->slurk", Gi, As[j])
    return [np.ascontiguousarray(a) for a in As]


def decoupled_chain_tensors(d: int, D: int, seed: int, axis: int = 0):
    """Four sites whose legs across one axis carry only index 0, so that
    every row (axis 0) or column (axis 1) of the lattice is an independent
    infinite matrix-product state.  a_i ~ N(0, 1) (seed; sites in index
    order), d x D x D [s, from, to]:
      axis 0: A[s, l, 0, r, 0] = a_i[s, l, r]  (rows, tensors a_(0,y), a_(1,y))
      axis 1: A[s, 0, u, 0, d] = a_i[s, d, u]  (columns, a_(x,0), a_(x,1))
    zero elsewhere.  Returns (As, a)."""
    rng = np.random.default_rng(seed)
    a = [rng.standard_normal((d, D, D)) for _ in range(4)]
    As = []
    for t in a:
        A = np.zeros((d, D, D, D, D))
        if axis == 0:
            A[:, :, 0, :, 0] = t
        else:
            A[:, 0, :, 0, :] = t.transpose(0, 2, 1)
        As.append(A)
    return As, a


# --------------------------------------------------------------------------
# environments
# --------------------------------------------------------------------------
def env_shapes(chi: int, D: int):
    c = (chi, chi)
    t = (chi, D, D, chi)
    return {"C1": c, "T1": t, "C2": c, "T2": t, "C3": c, "T3": t, "C4": c, "T4": t}


def random_env(chi: int, Ds, seed: int, per_site: bool = False):
    """Random initial C/T for every site.

    ``Ds[i]`` is the bond dimension around site i.  One
    ``default_rng(seed)`` stream; per tensor in the order C1, C2, C3, C4,
    T1, T2, T3, T4, standard normal in C order.  Each T is symmetrised over
    (k, k') so that the bra and ket layers of the network stay
    interchangeable.  By default one draw is shared by every site (all Ds
    equal): independent per-site starts can lock different sites of a
    symmetric network into inconsistent sectors, which the iteration does
    not always undo.  ``per_site=True`` draws each site in index order.
    """
    rng = np.random.default_rng(seed)

    def draw(D):
        sh = env_shapes(chi, D)
        e = {}
        for name in ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4"):
            e[name] = rng.standard_normal(sh[name])
        for name in ("T1", "T2", "T3", "T4"):
            T = e[name]
            e[name] = 0.5 * (T + T.transpose(0, 2, 1, 3))
        return {k: np.ascontiguousarray(v) for k, v in e.items()}

    if per_site:
        return [draw(D) for D in Ds]
    if len(set(Ds)) != 1:
        raise ValueError("a shared start needs one bond dimension")
    e0 = draw(Ds[0])
    return [{k: v.copy() for k, v in e0.items()} for _ in Ds]


# --------------------------------------------------------------------------
# operators (model definitions, Sec. 5.1 and the element example of Sec. 5.2)
# --------------------------------------------------------------------------
def spin_ops(d: int):
    """Spin-S matrices, S=(d-1)/2, basis m = S, S-1, ..., -S (index 0 = up)."""
    S = (d - 1) / 2.0
    m = S - np.arange(d)
    Sz = np.diag(m)
    Sp = np.zeros((d, d))
    for k in range(1, d):
        # S+ |m_k> = sqrt(S(S+1) - m_k(m_k+1)) |m_k + 1> ; m_{k-1} = m_k + 1
        Sp[k - 1, k] = np.sqrt(S * (S + 1) - m[k] * (m[k] + 1))
    Sm = Sp.T.copy()
    Sx = 0.5 * (Sp + Sm)
    return {"Sz": Sz, "Sp": Sp, "Sm": Sm, "Sx": Sx, "Id": np.eye(d)}


def boson_ops(nmax: int):
    d = nmax + 1
    b = np.zeros((d, d))
    for n in range(1, d):
        b[n - 1, n] = np.sqrt(n)
    return {"b": b, "bdag": b.T.copy(), "n": np.diag(np.arange(d, dtype=np.float64)),
            "Id": np.eye(d)}


def heisenberg_bond(d: int = 2):
    """S_i.S_j = Sz Sz + (S+ S- + S- S+)/2 on the combined index."""
    o = spin_ops(d)
    return (np.kron(o["Sz"], o["Sz"])
            + 0.5 * (np.kron(o["Sp"], o["Sm"]) + np.kron(o["Sm"], o["Sp"])))


def blbq_bond(d: int = 3, J: float = 1.0, K: float = 0.1):
    """Bilinear-biquadratic J S.S + K (S.S)^2 (Sec. 5.1, B = K)."""
    SS = heisenberg_bond(d)
    return J * SS + K * (SS @ SS)


def tfim_bond(d: int = 2, Jz: float = -1.0):
    o = spin_ops(d)
    return Jz * np.kron(o["Sz"], o["Sz"])


def boson_bond(nmax: int = 2, t: float = 0.1, V: float = 1.0):
    o = boson_ops(nmax)
    hop = np.kron(o["bdag"], o["b"]) + np.kron(o["b"], o["bdag"])
    return -t * hop + V * np.kron(o["n"], o["n"])


# The element listing of the S=1/2 Heisenberg bond given in Sec. 5.2:
# (i_before, j_before, i_after, j_after, re, im)
HEISENBERG_ELEMENTS_EXAMPLE = (
    (0, 0, 0, 0, 0.25, 0.0),
    (1, 0, 1, 0, -0.25, 0.0),
    (0, 1, 1, 0, 0.5, 0.0),
    (1, 0, 0, 1, 0.5, 0.0),
    (0, 1, 0, 1, -0.25, 0.0),
    (1, 1, 1, 1, 0.25, 0.0),
)

# Nearest-neighbour bonds of the 2x2 square cell, (source site, dx, dy) (Sec. 5.2)
SQUARE_2X2_BONDS = ((0, 0, 1), (0, 1, 0), (1, 0, 1), (1, 1, 0),
                    (2, 0, 1), (2, 1, 0), (3, 0, 1), (3, 1, 0))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def workload(name: str):
    """Return dict(As, envs, chi, d, D, sweeps, ops...) for a named workload."""
    if name == "neel_d2_D3_chi16":
        d, D, chi = 2, 3, 16
        As = neel_tensors(d, D, 0.1, seed=0)
        envs = random_env(chi, [D] * 4, seed=1)
        return dict(As=As, envs=envs, chi=chi, d=d, D=D, sweeps=50,
                    op1=spin_ops(2)["Sz"], op2=heisenberg_bond(2))
    if name == "neel_d2_D6_chi72":
        d, D, chi = 2, 6, 72
        As = neel_tensors(d, D, 0.1, seed=2)
        envs = random_env(chi, [D] * 4, seed=3)
        return dict(As=As, envs=envs, chi=chi, d=d, D=D, sweeps=100,
                    op1=spin_ops(2)["Sz"], op2=heisenberg_bond(2))
    if name == "xpol_d3_D8_chi128":
        d, D, chi = 3, 8, 128
        As = x_polarised_tensors(d, D, 0.05, seed=3)
        envs = random_env(chi, [D] * 4, seed=4)
        return dict(As=As, envs=envs, chi=chi, d=d, D=D, sweeps=20,
                    op1=spin_ops(3)["Sx"], op2=blbq_bond(3, 1.0, 0.1))
    raise KeyError(name)


def serving_request(j: int, ds=(2, 3), Ds=(4, 6, 8), chis=(32, 64, 128)):
    """Request j of the serving workload (a field / coupling scan family):
    d, D, chi drawn from seed 10000 + j; d = 2: spin-1/2 polarised along +x
    with the transverse-field Ising bond; d = 3: soft-core bosons (n_max = 2)
    in the uniform state with the boson bond; product state + 0.05 N(0, 1)
    noise; random environment from the same seed."""
    rng = np.random.default_rng(10000 + j)
    d = int(rng.choice(ds))
    D = int(rng.choice(Ds))
    chi = int(rng.choice(chis))
    if d == 2:
        As = x_polarised_tensors(2, D, 0.05, seed=10000 + j)
        op1, op2 = spin_ops(2)["Sx"], tfim_bond(2)
    else:
        As = uniform_boson_tensors(2, D, 0.05, seed=10000 + j)
        op1, op2 = boson_ops(2)["n"], boson_bond(2)
    envs = random_env(chi, [D] * 4, seed=20000 + j)
    return dict(d=d, D=D, chi=chi, As=As, envs=envs, op1=op1, op2=op2)


def batch_instance(i: int):
    """Instance i of the batched workload (64 uneven instances): seed 100 + i
    draws D in {3, 4, 5, 6}, then chi in {24, 32, 48, 64}; d = 2 Neel + 0.1
    N(0, 1) noise; environment from seed 200 + i."""
    rng = np.random.default_rng(100 + i)
    D = int(rng.choice((3, 4, 5, 6)))
    chi = int(rng.choice((24, 32, 48, 64)))
    As = neel_tensors(2, D, 0.1, seed=100 + i)
    envs = random_env(chi, [D] * 4, seed=200 + i)
    return dict(d=2, D=D, chi=chi, As=As, envs=envs, op1=spin_ops(2)["Sz"], op2=heisenberg_bond(2))

