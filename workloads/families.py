"""Generator families of permutation Cayley graphs, as plain one-line lists.

A permutation on {0..n-1} is a list ``p`` of length n with ``p[i]`` the image of ``i``.
Cycle notation ``(a b c)`` is the map a->b, b->c, c->a (0-based, as in the paper's
tables of maximal diameters, Section 3.4, and its generator definitions, Section 3.7).

The growth of a Cayley graph does not depend on whether a generator acts on states by
gather, by scatter, or by left multiplication (Section 2.1: growth is a property of the
group and generating set; the word map w -> w^-1 is a length-preserving bijection between
words over S and words over S^-1).  The families below therefore only fix the set S.

Family definitions follow the naming list of Section 3.3 ("Generators naming"):
Coxeter, cyclic Coxeter, LX/LRX, all transpositions, star (1,i), 3-cycles, (01i) with
inverses, consecutive 3-cycles with inverses, prefix cycles, pancake, reversals and
transposons (Section 5.2), plus the Koltsov3involutions construction of Section 3.7.
"""

from __future__ import annotations

import re
from typing import Callable, Dict, List, Sequence

import numpy as np

Perm = List[int]


def identity(n: int) -> Perm:
    return list(range(n))


def from_cycles(n: int, text: str) -> Perm:
    """Parse cycle notation such as ``(01)(23)`` or ``(1,11,9,10)(04)`` into one-line form.

    Inside a pair of parentheses, entries are comma separated when any is multi-digit,
    otherwise every character is one single-digit entry (the paper's tables use both).
    """
    p = list(range(n))
    for body in re.findall(r"\(([^)]*)\)", text):
        body = body.strip()
        if "," in body:
            cyc = [int(t) for t in body.split(",") if t.strip() != ""]
        else:
            cyc = [int(ch) for ch in body if not ch.isspace()]
        if len(set(cyc)) != len(cyc) or any(c < 0 or c >= n for c in cyc):
            raise ValueError(f"bad cycle ({body}) for n={n}")
        for a, b in zip(cyc, cyc[1:] + cyc[:1]):
            p[a] = b
    return p


def compose(p: Sequence[int], q: Sequence[int]) -> Perm:
    """The map x -> p[q[x]] (apply q first)."""
    return [p[q[x]] for x in range(len(p))]


def inverse(p: Sequence[int]) -> Perm:
    inv = [0] * len(p)
    for i, v in enumerate(p):
        inv[v] = i
    return inv


def is_inverse_closed(gens: Sequence[Sequence[int]]) -> bool:
    s = {tuple(g) for g in gens}
    return all(tuple(inverse(g)) in s for g in gens)


def inverse_closure(gens: Sequence[Sequence[int]]) -> List[Perm]:
    """Append each generator's inverse unless already present; drop identities.

    This is the "inverses appended" reading for random generator sets: involutions add
    nothing and the identity contributes no edges.
    """
    out: List[Perm] = []
    seen = set()
    for g in list(gens) + [inverse(g) for g in gens]:
        t = tuple(g)
        if t == tuple(range(len(g))) or t in seen:
            continue
        seen.add(t)
        out.append(list(g))
    return out


def transposition(n: int, i: int, j: int) -> Perm:
    p = list(range(n))
    p[i], p[j] = p[j], p[i]
    return p


def cycle(n: int, elems: Sequence[int]) -> Perm:
    p = list(range(n))
    for a, b in zip(elems, list(elems[1:]) + [elems[0]]):
        p[a] = b
    return p


# --- families of Section 3.3 ------------------------------------------------------------

def coxeter(n: int) -> List[Perm]:
    """Adjacent transpositions (i, i+1), i = 0..n-2."""
    return [transposition(n, i, i + 1) for i in range(n - 1)]


def cyclic_coxeter(n: int) -> List[Perm]:
    """Coxeter generators plus the wrap-around transposition (0, n-1)."""
    return coxeter(n) + ([transposition(n, 0, n - 1)] if n > 2 else [])


def all_transpositions(n: int) -> List[Perm]:
    return [transposition(n, i, j) for i in range(n) for j in range(i + 1, n)]


def star(n: int) -> List[Perm]:
    """Transpositions (0, i), i = 1..n-1 (the star graph)."""
    return [transposition(n, 0, i) for i in range(1, n)]


def _left_shift(n: int) -> Perm:
    return [(i + 1) % n for i in range(n)]


def lrx(n: int) -> List[Perm]:
    """L = cyclic left shift, R = L^-1, X = swap of positions 0 and 1."""
    L = _left_shift(n)
    return [L, inverse(L), transposition(n, 0, 1)]


def lx(n: int) -> List[Perm]:
    """L and X only (directed, not inverse-closed for n > 2)."""
    return [_left_shift(n), transposition(n, 0, 1)]


def pancake(n: int) -> List[Perm]:
    """Prefix reversals of lengths 2..n (involutions)."""
    gens = []
    for j in range(2, n + 1):
        gens.append([j - 1 - i if i < j else i for i in range(n)])
    return gens


def reversals(n: int) -> List[Perm]:
    """All segment reversals r_{i,j}, 0 <= i < j <= n-1 (Section 5.2, |R| = C(n,2))."""
    gens = []
    for i in range(n):
        for j in range(i + 1, n):
            p = list(range(n))
            p[i:j + 1] = p[i:j + 1][::-1]
            gens.append(p)
    return gens


def transposons(n: int) -> List[Perm]:
    """Block transpositions: exchange adjacent blocks [i, j) and [j, k), 0 <= i < j < k <= n."""
    gens = []
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n + 1):
                order = list(range(i)) + list(range(j, k)) + list(range(i, j)) + list(range(k, n))
                gens.append(order)
    return gens


def three_cycles(n: int) -> List[Perm]:
    """All 3-cycles (both orientations); they generate A_n."""
    gens = []
    for a in range(n):
        for b in range(n):
            for c in range(n):
                if a < b and a < c and b != c:
                    gens.append(cycle(n, [a, b, c]))
    return gens


def cycles_01i_inv(n: int) -> List[Perm]:
    """3-cycles (0, 1, i), i = 2..n-1, with their inverses ("(01i)I")."""
    return inverse_closure([cycle(n, [0, 1, i]) for i in range(2, n)])


def consecutive_3cycles_inv(n: int) -> List[Perm]:
    """Consecutive 3-cycles (i, i+1, i+2) with inverses ("(i,i+1,i+2)I")."""
    return inverse_closure([cycle(n, [i, i + 1, i + 2]) for i in range(n - 2)])


def prefix_cycles(n: int) -> List[Perm]:
    """Prefix cycles (0, 1, ..., i), i = 1..n-1 (directed)."""
    return [cycle(n, list(range(i + 1))) for i in range(1, n)]


def consecutive_4cycles(n: int) -> List[Perm]:
    """Consecutive 4-cycles (i, i+1, i+2, i+3), i = 0..n-4 (directed; Section 3.2, acting on
    binary vectors)."""
    return [cycle(n, [i, i + 1, i + 2, i + 3]) for i in range(n - 3)]


def binary_start(n: int) -> List[int]:
    """Central state of the "Bin" coset S_n / (S_m x S_{n-m}), m = floor(n/2): m zeros, then
    ones (Section 3.2 and the Schreier-graph table)."""
    m = n // 2
    return [0] * m + [1] * (n - m)


def koltsov3(n: int, type_: int, k: int, d: int = 1) -> List[Perm]:
    """Koltsov3involutions (Section 3.7): I = prod_{i even}(i,i+1), K = prod_{i odd}(i,i+1),
    and S = (k, k+d) for type 1 or S = (k, k+3)(k+1, k+2) for type 2."""
    I = list(range(n))
    K = list(range(n))
    for i in range(0, n - 1):
        tgt = I if i % 2 == 0 else K
        tgt[i], tgt[i + 1] = tgt[i + 1], tgt[i]
    if type_ == 1:
        S = transposition(n, k, k + d)
    elif type_ == 2:
        S = list(range(n))
        S[k], S[k + 3] = S[k + 3], S[k]
        S[k + 1], S[k + 2] = S[k + 2], S[k + 1]
    else:
        raise ValueError("type must be 1 or 2")
    return [I, K, S]


def random_perms(rng: np.random.Generator, n: int, k: int) -> List[Perm]:
    """k uniformly random non-identity permutations of {0..n-1} (rejection of the identity)."""
    gens = []
    ident = list(range(n))
    while len(gens) < k:
        p = [int(x) for x in rng.permutation(n)]
        if p != ident:
            gens.append(p)
    return gens


FAMILIES: Dict[str, Callable[[int], List[Perm]]] = {
    "coxeter": coxeter,
    "cyclic_coxeter": cyclic_coxeter,
    "all_transpositions": all_transpositions,
    "star": star,
    "lrx": lrx,
    "lx": lx,
    "pancake": pancake,
    "reversals": reversals,
    "transposons": transposons,
    "three_cycles": three_cycles,
    "cycles_01i_inv": cycles_01i_inv,
    "consecutive_3cycles_inv": consecutive_3cycles_inv,
    "prefix_cycles": prefix_cycles,
    "consecutive_4cycles": consecutive_4cycles,
}
