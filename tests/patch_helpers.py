"""Cut a patch out of a large mesh for the oracle: the elements within a
graph distance of some seed elements, as a standalone mesh whose faces to
elements outside the patch become walls.  A result of the discrete scheme
at a seed element depends only on the elements within its domain of
dependence: one operator application reaches the face neighbours (distance
1), the predictor is element-local, one ADER step reaches distance 1 and
one five-stage LSRK step distance 5.  So with a radius at least that large,
the oracle on the patch gives the seed elements' results exactly."""
import numpy as np


def patch(mesh, rho, c, U, seeds, radius):
    nbr = np.asarray(mesh["nbr"])
    seen = {int(e): 0 for e in seeds}
    frontier = [int(e) for e in seeds]
    for r in range(radius):
        nxt = []
        for e in frontier:
            for f in range(6):
                en = int(nbr[e, f])
                if en >= 0 and en not in seen:
                    seen[en] = r + 1
                    nxt.append(en)
        frontier = nxt
    ids = np.array(sorted(seen), np.int64)
    pos = {int(e): i for i, e in enumerate(ids)}
    sub_nbr = np.array([[pos.get(int(nbr[e, f]), -1) if nbr[e, f] >= 0 else -1 for f in range(6)]
                        for e in ids], np.int32)
    sub = {"n_elem": len(ids), "geom_degree": mesh["geom_degree"],
           "nodes": np.asarray(mesh["nodes"])[ids], "nbr": sub_nbr,
           "nbr_face": np.asarray(mesh["nbr_face"])[ids], "orient": np.asarray(mesh["orient"])[ids]}
    return sub, ids, np.asarray(rho)[ids], np.asarray(c)[ids], np.asarray(U)[ids], [pos[int(s)] for s in seeds]
