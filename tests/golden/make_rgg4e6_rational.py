"""Write rgg4e6_rational_psi.txt: FP64 oracle values for the full-size
rational-Krylov probing check (Section 3.1 probing vectors, eq.
rational-krylov-approximation-quadform with the poles of Section 4.2).

Input: the random geometric graph n = 4e6 in the unit square, radius
sqrt(6 / (pi n)), seed 4; rho = L / tr L.  Colouring: the oracle's greedy
distance-2 colouring (Algorithm 1).  For colour classes 0..3 the oracle
evaluates psi = v^T f(A) v by rational Krylov with the default 8 poles and
2 poles at infinity, each shifted system solved by conjugate gradients to a
relative residual of 1e-10.  Each line: colour, class size, the sum of the
class's node ids, the sum of their squares (so that a test can check it has
the same class), psi.

Run (calls only the oracle and the seeded input generator):
    python tests/golden/make_rgg4e6_rational.py
"""
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, SEED, COLOURS = 4_000_000, 4, 4
OUT = os.path.join(HERE, "rgg4e6_rational_psi.txt")


def _graph():
    from paper_2212_09642_gb300 import graphs
    return graphs.random_geometric(N, graphs.rgg_radius_for_degree(N, 6), SEED)


def _psi(job):
    colour, nodes = job
    import numpy as np
    from oracle import density, rational
    g = _graph()
    A, _ = density.density_matrix(g)
    v = np.zeros(g.n)
    v[nodes] = 1.0
    t = time.time()
    psi = rational.rational_quadform(A, v, rational.default_shifts(A), n_inf=2, method="cg")
    return colour, psi, time.time() - t


def main():
    import numpy as np
    from oracle import coloring
    t0 = time.time()
    g = _graph()
    col = coloring.greedy_distance_coloring(g, 2)
    print(f"colouring: {int(col.max()) + 1} colours in {time.time() - t0:.0f} s", flush=True)
    jobs = [(c, np.nonzero(col == c)[0]) for c in range(COLOURS)]
    with mp.get_context("spawn").Pool(COLOURS) as pool:
        res = pool.map(_psi, jobs)
    with open(OUT, "w") as fh:
        fh.write("# written by tests/golden/make_rgg4e6_rational.py (oracle only); RGG n=4e6 r=sqrt(6/(pi n)) "
                 "seed 4, greedy distance-2 colouring (Algorithm 1), rational Krylov psi of colour classes "
                 "0..3, default 8 poles + 2 at infinity, CG to 1e-10\n")
        fh.write(f"# colours in the distance-2 colouring: {int(col.max()) + 1}\n")
        fh.write("# colour size id_sum id_square_sum psi\n")
        for (c, nodes), (_, psi, dt) in zip(jobs, res):
            ids = nodes.astype(np.int64)
            fh.write(f"{c} {ids.size} {int(ids.sum())} {int((ids * ids).sum())} {psi:.17g}\n")
            print(f"colour {c}: {ids.size} nodes, psi {psi:.17g} ({dt:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
