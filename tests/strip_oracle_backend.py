"""A host backend for the strip protocol (test code only): each strip's
directions, local counts, exit numbers and final counts computed by the
oracle, so that the partition, the exchanges and the link solve of
paper_1605_05773_gb300.strips run on CPU and are checked against the oracle
on the whole grid."""
import numpy as np
import torch

import oracle


class OracleStrips:
    def __init__(self, rule="steepest"):
        self.rule = rule

    def directions(self, z_ext, halo):
        top, bot = halo & 1, (halo >> 1) & 1
        h = z_ext.shape[0] - top - bot
        d = oracle.flowdir(z_ext.cpu().numpy(), self.rule)  # the halo rows are the array's own edge rows
        return torch.from_numpy(np.ascontiguousarray(d[top:top + h]))

    def local_counts(self, dir):
        return torch.from_numpy(oracle.accumulate(dir.cpu().numpy()))

    def exit_numbers(self, dir, c):
        G = oracle.transposed(dir.cpu().numpy(), c.cpu().numpy().astype(np.float64))
        return torch.from_numpy(G.astype(np.float32))

    def final_counts(self, dir, top_in, bottom_in):
        d = dir.cpu().numpy()
        w = np.ones(d.shape, dtype=np.float64)
        if top_in is not None:
            w[0] += top_in.cpu().numpy().astype(np.float64)
        if bottom_in is not None:
            w[-1] += bottom_in.cpu().numpy().astype(np.float64)
        return torch.from_numpy(np.rint(oracle.accumulate_weighted(d, w)).astype(np.uint32))
