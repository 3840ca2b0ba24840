"""Autotuner of psgld_batch_sweep's launch knobs.

The knobs it searches change how work is spread over the GPU, never what is
computed: `batch_ctas` (CTAs of each persistent two-sided batch launch; every
item is computed by one CTA whichever CTA takes it) and `batch_update_blocks`
(blocks of each batch update launch, a grid-stride loop over the items).  So
a chain ends in the same state, bit for bit, whatever the tuner tries or
chooses, and the sweeps the tuner times are ordinary sweeps of the chains
(they count toward the chains' iterations, and burn-in, as any other).

tune_batch() times each candidate with CUDA events over a few batched
sweeps, one knob at a time (CTAs first, with the default update grid, then
the update grid with the chosen CTAs), sets the fastest on the list's first
context (which the library reads the knobs from) and returns the choice with
every timing, so that a caller can record it.
"""
from __future__ import annotations

from . import psgld as P

CTA_CANDIDATES = (0, 144, 128, 112, 96, 76)          # 0: one CTA per SM
UPDATE_BLOCK_CANDIDATES = (0, 152 * 4, 152 * 8, 152 * 32)   # 0: one per 256 items, at most 2432


def _time_sweeps(chains, sweeps, stream):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    P.psgld_batch_sweep(chains, sweeps, stream.cuda_stream)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / sweeps


def tune_batch(chains, sweeps_per_trial: int = 2, repeats: int = 2,
               cta_candidates=CTA_CANDIDATES, update_candidates=UPDATE_BLOCK_CANDIDATES):
    """Tune the batch launch knobs for `chains` (P.PSGLD objects, the list a
    caller passes to psgld_batch_sweep).  Runs (len(cta_candidates) +
    len(update_candidates)) * repeats * sweeps_per_trial sweeps, plus one
    untimed sweep per knob setting (its graph capture).  Returns
    {"batch_ctas": c, "batch_update_blocks": u, "ms_per_sweep": {...}}."""
    import torch
    stream = torch.cuda.current_stream()
    lead = chains[0]
    timings = {}

    def trial(ctas, blocks):
        lead.set_options(batch_ctas=ctas, batch_update_blocks=blocks)
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)        # capture (untimed)
        best = min(_time_sweeps(chains, sweeps_per_trial, stream) for _ in range(repeats))
        timings[f"ctas={ctas},update_blocks={blocks}"] = best
        return best

    ctas = min(cta_candidates, key=lambda c: trial(c, 0))
    blocks = min(update_candidates, key=lambda u: trial(ctas, u) if u else
                 timings[f"ctas={ctas},update_blocks=0"])
    lead.set_options(batch_ctas=ctas, batch_update_blocks=blocks)
    return {"batch_ctas": ctas, "batch_update_blocks": blocks, "ms_per_sweep": timings,
            "knobs": "batch_ctas: CTAs of each persistent two-sided batch launch (0: one per "
                     "SM); batch_update_blocks: blocks of each batch update launch (0: one per "
                     "256 items, at most 2432); neither changes any result"}
