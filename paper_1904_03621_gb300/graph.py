"""Dictionary-graph front end in the style of the paper's Python wrapper (Sec. 4.1).

The paper's package takes the problem as a graph -- a dict mapping node pairs to
weights, a pair (i, i) giving the field of node i -- and a number of states, and
returns their energies and states.  `search` does the same on top of the CUDA
library: it orders the node labels, builds the dense coupling matrix and field
vector (argument marshalling only) and calls `api.low_spectrum` (Ising, Eq. (1)) or
`api.low_spectrum_qubo` (QUBO, Eqs. (2)-(3)).  Energies follow the library's sign,
E = +sum J s s + sum h s; pass the negated weights to obtain the paper's H.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Solution:
    energies: np.ndarray       # (S,) ascending; int64 for integer weights, float64 otherwise
    states: np.ndarray         # (S, n) spins +-1 (Ising) or 0/1 (QUBO), columns in `nodes` order
    configurations: np.ndarray  # (S,) uint64, bit k = node k is +1 (Ising) or 1 (QUBO)
    nodes: list                # node labels in column / bit order


def graph_to_dense(graph: dict, dtype=None):
    """Dense (J, h, nodes) of a dict graph.

    Nodes are the sorted labels that appear in any key.  Key (i, i) adds to the field of
    i; key (i, j), i != j, adds to the coupling of the unordered pair (written to the
    upper triangle, so (i, j) and (j, i) accumulate).  dtype defaults to int32 when every
    weight is an integer, float64 otherwise.
    """
    if not graph:
        raise ValueError("empty graph")
    nodes = sorted({v for key in graph for v in key})
    index = {v: k for k, v in enumerate(nodes)}
    n = len(nodes)
    if dtype is None:
        dtype = np.int32 if all(isinstance(w, (int, np.integer)) for w in graph.values()) else np.float64
    J = np.zeros((n, n), dtype=np.float64)
    h = np.zeros(n, dtype=np.float64)
    for (u, v), w in graph.items():
        i, j = index[u], index[v]
        if i == j:
            h[i] += w
        else:
            J[min(i, j), max(i, j)] += w
    return J.astype(dtype), h.astype(dtype), nodes


def search(graph: dict, num_states: int, *, qubo: bool = False, dtype=None, device="cuda", **options) -> Solution:
    """The `num_states` lowest states of the model the graph defines (exhaustive, exact).

    qubo=False: Ising spins s in {-1, +1}, E(s) = sum J_ij s_i s_j + sum h_i s_i.
    qubo=True:  binary q in {0, 1},      F(q) = sum a_ij q_i q_j + sum b_i q_i.
    Extra keyword options go to the library call (variant, fixed_bits, ...).
    """
    import torch

    from . import api

    J, h, nodes = graph_to_dense(graph, dtype)
    Jt = torch.from_numpy(np.ascontiguousarray(J)).to(device)
    ht = torch.from_numpy(np.ascontiguousarray(h)).to(device)
    if qubo:
        e, st = api.low_spectrum_qubo(Jt, ht, num_states, **options)
    else:
        e, st = api.low_spectrum(Jt, ht, num_states, **options)
    conf = api.states_u64(st)
    n = len(nodes)
    bits = ((conf[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.int8)
    states = bits if qubo else (2 * bits - 1).astype(np.int8)
    return Solution(energies=e.cpu().numpy(), states=states, configurations=conf, nodes=nodes)
