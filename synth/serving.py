"""Seeded synthetic serving load (inputs only): many independent planted
PARAFAC2 streams whose update batches arrive as one Poisson process.

Each stream is a planted stream of `synth.planted` (the same recipe: U(0,1)
factors, orthonormal Q_k drawn at the final length, absolute noise σ) with
its own J, R and initial slice count, and with serving-style updates: each
update touches a random fraction f ~ U(0, 1] of the stream's slices with
U{1..256} new rows each and adds U{0..50} new slices of U{1..256} rows.
Update batches of all streams arrive as one Poisson process of a given total
rate; each arrival belongs to a stream drawn uniformly.  The module draws
numbers and multiplies out planted factors; it holds none of Dash's
arithmetic.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import torch

from synth.planted import BASE_SEED, Workload

SERVING_SEED = BASE_SEED + 4


@dataclasses.dataclass
class ServingLoad:
    """Streams and their update arrivals.

    streams[s] is stream s's workload (batch 0 = its initial tensor);
    arrivals lists (time in s, stream, update index t >= 1) in time order,
    the t-th arrival of a stream being its update t."""
    streams: List[Workload]
    arrivals: List[Tuple[float, int, int]]

    def updates_of(self, s: int) -> int:
        return self.streams[s].steps


def serving_load(n_streams: int = 64, duration: float = 10.0, rate: float = 2000.0,
                 J_choices: Sequence[int] = (64, 128, 256), R_choices: Sequence[int] = (8, 16, 32),
                 K0_range: Tuple[int, int] = (500, 10000), init_rows: Tuple = ("uniform", 50, 400),
                 rows: Tuple = ("uniform", 1, 256), new_slices: Tuple = ("uniform", 0, 50),
                 new_rows: Tuple = ("uniform", 1, 256), touch: Tuple = ("uniform", 0.0, 1.0),
                 sigma: float = 0.1, lam: float = 0.95, seed: int = SERVING_SEED) -> ServingLoad:
    """The serving workload: n_streams planted streams, Poisson arrivals of
    total mean `rate` per second over `duration` seconds."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    arrivals: List[Tuple[float, int, int]] = []
    count = [0] * n_streams
    t = 0.0
    while True:
        u = float(torch.rand(1, generator=g, dtype=torch.float64))
        t += -math.log(max(u, 1e-300)) / rate
        if t > duration:
            break
        s = int(torch.randint(0, n_streams, (1,), generator=g))
        count[s] += 1
        arrivals.append((t, s, count[s]))
    streams = []
    for s in range(n_streams):
        J = int(J_choices[int(torch.randint(0, len(J_choices), (1,), generator=g))])
        R = int(R_choices[int(torch.randint(0, len(R_choices), (1,), generator=g))])
        K0 = int(torch.randint(K0_range[0], K0_range[1] + 1, (1,), generator=g))
        streams.append(Workload(name=f"serve{s}", K0=K0, J=J, R=R, init_rows=init_rows,
                                steps=count[s], rows_per_step=rows, new_slices_per_step=0,
                                new_slice_rows=new_rows, sigma=sigma, lam=lam,
                                seed=seed + 1 + s, touch=touch, new_slices_dist=new_slices))
    return ServingLoad(streams=streams, arrivals=arrivals)
