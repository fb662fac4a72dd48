"""Converts factors between the oracle's Factorization and the library's mht_factors arrays.

Test-only glue: the oracle and the library share no code; this module only reshapes arrays.
"""
import numpy as np

from oracle import butterfly as B


def oracle_to_arrays(F: B.Factorization) -> dict:
    nb = 1 << F.L
    ranks = np.concatenate([np.asarray(F.ranks[l], dtype=np.int32) for l in range(F.L + 1)])
    perms = [np.asarray(p, dtype=np.int32) for l in range(F.L + 1) for p in F.perms[l]]
    Ts = [np.asarray(t).ravel() for l in range(F.L + 1) for t in F.T[l]]
    Us = [np.asarray(u).ravel() for u in F.U]
    dt = np.complex128 if F.complex_ else np.float64
    return {
        "n": F.n, "m": F.m, "levels": F.L, "complex": F.complex_,
        "space_perm": F.space_perm, "space_offsets": F.space_off,
        "mode_perm": F.mode_perm, "mode_offsets": F.mode_off,
        "ranks": ranks,
        "local_perm": np.concatenate(perms) if perms else np.zeros(0, np.int32),
        "transfer": np.concatenate(Ts).astype(dt) if Ts else np.zeros(0, dt),
        "column_bases": np.concatenate(Us).astype(dt) if Us else np.zeros(0, dt),
        "nb": nb,
    }


def arrays_to_oracle(d: dict) -> B.Factorization:
    L = int(d["levels"])
    nb = 1 << L
    F = B.Factorization(L, int(d["n"]), int(d["m"]), bool(d["complex"]),
                        np.asarray(d["space_perm"]), np.asarray(d["space_offsets"]),
                        np.asarray(d["mode_perm"]), np.asarray(d["mode_offsets"]))
    ranks = np.asarray(d["ranks"]).reshape(L + 1, nb)
    pp = tp = 0
    for l in range(L + 1):
        F.ranks.append(ranks[l].astype(np.int64))
        pl, tl = [], []
        for b in range(nb):
            K = F.block_input_size(l, b)
            r = int(ranks[l][b])
            pl.append(np.asarray(d["local_perm"][pp:pp + K], dtype=np.int64))
            pp += K
            tl.append(np.asarray(d["transfer"][tp:tp + r * (K - r)]).reshape(r, K - r))
            tp += r * (K - r)
        F.perms.append(pl)
        F.T.append(tl)
    up = 0
    for t in range(nb):
        rows = int(F.space_off[t + 1] - F.space_off[t])
        r = int(ranks[L][t])
        F.U.append(np.asarray(d["column_bases"][up:up + rows * r]).reshape(rows, r))
        up += rows * r
    return F
