"""Request loop over :class:`paper_2010_06931_gb300.Server`: Poisson
arrivals, continuous batching, per-request latency.

Requests arrive at exponentially distributed intervals; each arrival is
submitted at once, the server steps (admits what fits, retires what is
finished; the solves themselves run on the device without the host) and
every finished request is polled out immediately.  Latency = completion
time - arrival time (queueing, admission and solve).
"""
import time

import numpy as np

from . import Server


def serve_poisson(server, requests, rate_hz, seed=0, poll_every=1):
    """Runs the arrival process over ``requests`` (dicts of Server.submit
    arguments).  Returns a dict with per-request latencies (s), results,
    stats and the wall time."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=len(requests)))
    arrivals -= arrivals[0]
    t0 = time.perf_counter()
    pending = {}  # ticket -> request index
    nxt = 0
    lat = [None] * len(requests)
    out = [None] * len(requests)
    stats = [None] * len(requests)
    steps = 0
    while nxt < len(requests) or pending:
        now = time.perf_counter() - t0
        while nxt < len(requests) and arrivals[nxt] <= now:
            pending[server.submit(**requests[nxt])] = nxt
            nxt += 1
        if not pending:
            time.sleep(max(0.0, min(0.01, arrivals[nxt] - now)))
            continue
        active, _ = server.step()
        steps += 1
        finished = 0
        if steps % poll_every == 0 or active == 0:
            for tk in list(pending):
                if server.state(tk) == Server.DONE:
                    k = pending.pop(tk)
                    _, out[k], stats[k], rc = server.poll(tk)
                    lat[k] = time.perf_counter() - t0 - arrivals[k]
                    stats[k] = dict(levels=stats[k], rc=rc)
                    finished += 1
        if active and not finished:
            time.sleep(2e-4)  # the solves run on the device; do not spin the host
    wall = time.perf_counter() - t0
    lat = np.array(lat)
    return dict(latency=lat, p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                wall=wall, pairs_per_s=len(requests) / wall, steps=steps, results=out, stats=stats,
                arrivals=arrivals)
