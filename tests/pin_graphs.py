"""Small hand-built graphs whose controller quantities (OPT^L, the LHGA order, the
approximation-ratio bound) are worked out by hand in test_oracle_controller.py; the
GPU tests run the same graphs through the library."""
import numpy as np

from paper_2405_12871_gb300 import synth


def graph(n, edges):
    edges = sorted(edges)
    src = [e[0] for e in edges]
    dst = [e[1] for e in edges]
    p = [e[2] for e in edges]
    return synth.csr_from_edges(n, src, dst, np.asarray(p, np.float32))


# seeds 0, 1; ON = {2, 3, 4, 5, 6, 9}; node 7 is a non-seed feeding node 2
OPT_EDGES = [
    (0, 1, 0.5),     # seed -> seed: not in ON
    (0, 2, 0.5), (1, 2, 0.25),   # q(2) = 1 - 0.5 * 0.75 = 0.625
    (0, 3, 0.75),                # q(3) = 0.75
    (1, 4, 0.5),                 # q(4) = 0.5
    (0, 5, 0.125),               # q(5) = 0.125
    (0, 6, 0.1), (1, 6, 0.1),    # q(6) = 1 - (1 - p_q(0.1))^2 ~ 0.19
    (0, 8, 0.0),                 # p = 0: never live, not in ON
    (1, 9, 0.0625),              # q(9) = 0.0625
    (7, 2, 0.5),                 # not from a seed: does not enter q(2)
]
OPT_N, OPT_S = 10, [0, 1]


def opt_graph():
    return graph(OPT_N, OPT_EDGES)


def lhga_graph():
    """Seed 0.  ON = {1, 2, 3, 4}:
      node 1: q = 0.25,  outdeg 4, indeg 1  -> score 1.0
      node 2: q = 0.5,   outdeg 2, indeg 1  -> score 1.0 (ties node 1; larger q)
      node 3: q = 0.75,  outdeg 1, indeg 3  -> score 0.75
      node 4: q = 0.125, outdeg 6, indeg 4  -> score 0.75
    Returns (graph, n)."""
    edges = [(0, 1, 0.25), (0, 2, 0.5), (0, 3, 0.75), (0, 4, 0.125)]
    sink = 5
    for u, d in ((1, 4), (2, 2), (3, 1), (4, 6)):
        for _ in range(d):
            edges.append((u, sink, 0.5))
            sink += 1
    # extra in-edges of nodes 3 and 4 from non-seed sinks (in-degree only)
    edges += [(5, 3, 0.5), (6, 3, 0.5), (7, 4, 0.5), (8, 4, 0.5), (9, 4, 0.5)]
    return graph(sink, edges), sink


# p = 1.  Seed 0 -> {1, 2, 3}; 1 -> {2, 3, 4}; 4 -> 5.  V'_s = {1, 2, 3, 4, 5}.
# LRR(t) inside R \ S: {1}, {1,2}, {1,3}, {1,4}, {1,4,5}: all contain node 1.
RATIO_EDGES = [(0, 1, 1.0), (0, 2, 1.0), (0, 3, 1.0), (1, 2, 1.0), (1, 3, 1.0), (1, 4, 1.0),
               (4, 5, 1.0)]


def ratio_graph():
    return graph(6, RATIO_EDGES)
