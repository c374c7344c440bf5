"""Schedule autotuning for the batched product (tft_polymul_batch).

A batch is split into two size classes at r = 2^small_log: the single-CTA
class below, the row/column class (one row length 2^lr, 2^clog columns per
column tile) above; within the row/column class the products whose columns
are shorter than the tallest get a column tile width of their own
(clog_lo), tuned after the rest.  The best split and row geometry depend on the batch's
length mix and on the device, so ``tune_batch`` times every admissible
schedule from a small candidate grid on the batch itself (plan once per
candidate, then CUDA-event timed runs) and returns the fastest.  Results
are cached per (prime, device name, SM count, length-mix signature) in a
JSON file next to the built library, so a serving process tunes each mix
once.

All transforms run in the CUDA library; this module only chooses the
``tft_batch_params`` it passes in.
"""

import json
import math
import os

from . import tft

_CACHE = os.path.join(os.path.dirname(tft.LIB_PATH), "batch_tune.json")


def candidates(prime):
    """The admissible grid of (small_log, lr, clog) for a prime."""
    pid = tft.prime_id(prime)
    small_max = 12 if pid == 2 else 13
    out = []
    for lr in range(8, 12):
        for small_log in range(max(lr, 9), small_max + 1):
            for clog in (2, 3, 4, 5):
                out.append({"small_log": small_log, "lr": lr, "clog": clog})
    return out


def mix_signature(lengths):
    """Histogram of ceil(log2 r) over the products (the length mix)."""
    h = {}
    for na, nb in lengths:
        r = int(na) + int(nb) - 1
        b = max(0, math.ceil(math.log2(r))) if r > 1 else 0
        h[b] = h.get(b, 0) + 1
    return ",".join(f"{k}:{h[k]}" for k in sorted(h))


def _key(ctx, lengths):
    import torch
    p = torch.cuda.get_device_properties(ctx.device)
    return f"{ctx.prime}|{p.name}|{p.multi_processor_count}|" + \
        mix_signature(lengths)


def _load_cache():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(c):
    tmp = _CACHE + f".{os.getpid()}.tmp"
    try:
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, _CACHE)
    except OSError:
        pass


def _column_classes(lengths, params):
    """Distinct column heights (padded, log2) among the products that take
    the row/column path under ``params``."""
    cs = set()
    for na, nb in lengths:
        r = int(na) + int(nb) - 1
        if r <= (1 << params["small_log"]):
            continue
        rows = -(-r // (1 << params["lr"]))
        cs.add((rows - 1).bit_length())
    return len(cs)


def time_schedule(ctx, products, params, reps=3, stream=None):
    """Mean milliseconds of one tft_batch_run of ``products`` planned with
    ``params`` (the batch reservation must already cover them)."""
    import torch
    s = stream or torch.cuda.current_stream()
    tft.tft_batch_plan(ctx, products, params)
    tft.tft_batch_run(ctx, s)  # warm-up
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        tft.tft_batch_run(ctx, s)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(ctx, products, reps=3, use_cache=True, grid=None):
    """Fastest schedule for ``products`` (a list of (a, b, out) CUDA
    tensors): returns (params, table) where table maps each tried schedule
    to its time in ms.  Reserves the batch work area for the largest
    candidate's need.  The outputs hold the last candidate's (correct)
    results afterwards."""
    lengths = [(a.numel(), b.numel()) for a, b, _ in products]
    key = _key(ctx, lengths)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit["params"]), hit.get("table", {})
    grid = grid or candidates(ctx.prime)
    need = max(tft.tft_batch_work_words(ctx.prime, lengths, g) for g in grid)
    tft.tft_ctx_reserve_batch(ctx, max(1, len(products)), need)
    table = {}
    best, best_ms = None, float("inf")
    for g in grid:
        try:
            ms = time_schedule(ctx, products, g, reps)
        except tft.TFTError as e:
            if e.status != tft.TFT_ERANGE:
                raise
            continue  # a product too long for this row length
        table["s{small_log}-lr{lr}-c{clog}".format(**g)] = ms
        if ms < best_ms:
            best, best_ms = g, ms
    if best is None:
        raise RuntimeError("no admissible batch schedule")
    # per size class: when the row/column products have columns of more
    # than one height, the shorter-column class runs its column passes as
    # launches of their own, and its tile width is tuned separately
    if _column_classes(lengths, best) > 1:
        for cl in range(0, min(5, best["lr"]) + 1):
            if cl == best["clog"]:
                continue
            g = dict(best, clog_lo=cl)
            try:
                ms = time_schedule(ctx, products, g, reps)
            except tft.TFTError as e:
                if e.status != tft.TFT_ERANGE:
                    raise
                continue
            table["s{small_log}-lr{lr}-c{clog}-clo{clog_lo}".format(**g)] = ms
            if ms < best_ms:
                best, best_ms = g, ms
    if use_cache:
        c = _load_cache()
        c[key] = {"params": best, "ms": best_ms, "table": table}
        _store_cache(c)
    return dict(best), table
