"""Seeded synthetic workloads (parameters and seeded draws only).

Each workload names the game variant, the search parameters and the seeds;
root states themselves are generated from `root_seed` by the engine's
dvc_init_states (and, in tests, independently by the oracle).  Budgets of the
uneven-forest workload are drawn log-uniformly with numpy from `seed`.
"""
from dataclasses import asdict, dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    nplayers: int
    ntiles: int
    deal: int
    max_predraw: int
    max_revealed: int
    playouts: int
    n_trees: int
    budget: int = 0            # fixed budget per tree (0: drawn)
    budget_lo: int = 0         # log-uniform range when drawn
    budget_hi: int = 0
    seed: int = 1              # search streams
    root_seed: int = 1         # root generation
    cont_thr: int = 1 << 31    # continue after a correct guess with probability 1/2 in playouts
    c_uct: float = 1.4142135623730951
    d_max: int = 8

    def budgets(self, n=None) -> np.ndarray:
        n = self.n_trees if n is None else n
        if self.budget:
            return np.full(n, self.budget, dtype=np.int32)
        rng = np.random.default_rng(self.seed)
        u = rng.uniform(np.log(self.budget_lo), np.log(self.budget_hi), size=self.n_trees)
        return np.floor(np.exp(u)).astype(np.int32)[:n]

    def config_kwargs(self):
        d = asdict(self)
        return {k: d[k] for k in ("nplayers", "ntiles", "deal", "max_predraw", "max_revealed", "cont_thr",
                                  "c_uct", "d_max", "playouts")}


# 2 players, 24 tiles, 4 dealt each (16 in the pool): one seeded deal,
# one tree, 10,000 iterations, one playout per leaf.
SINGLE_TREE = Workload("2p24_single_tree_10k", nplayers=2, ntiles=24, deal=4, max_predraw=0, max_revealed=5,
                       playouts=1, n_trees=1, budget=10000, seed=1, root_seed=1)

# 2 players, 24 tiles: 4,096 mid-game roots (0-10 post-deal draws, at most 5
# face-up tiles per player), 4,096 iterations x 256 playouts per tree
# (1,048,576 playouts per decision, 4.29e9 per batch).
BATCHED = Workload("2p24_4096trees_4096it_256po", nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5,
                   playouts=256, n_trees=4096, budget=4096, seed=2, root_seed=2)

# 4 players, 26 tiles with jokers, 3 dealt each (14 in the pool): 16,384
# trees with budgets log-uniform in [1k, 100k], 32 playouts per leaf.
UNEVEN = Workload("4p26_16384trees_loguniform_1k_100k_32po", nplayers=4, ntiles=26, deal=3, max_predraw=8,
                  max_revealed=3, playouts=32, n_trees=16384, budget_lo=1000, budget_hi=100000, seed=3, root_seed=3)

ALL = {w.name: w for w in (SINGLE_TREE, BATCHED, UNEVEN)}
