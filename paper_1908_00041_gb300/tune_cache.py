"""Persistent cache of the generator shapes chosen by the plan autotuner.

``favest_plan_tune`` times every generator shape the library offers on the plan's own
workload and keeps the fastest.  That takes from milliseconds to about a second per
plan.  The cache keeps the winner per (degree, batch, precision, I/O type, GPU name)
in a JSON file, so a later process applies it with ``favest_plan_set_gen_shape``
instead of timing again.

The file comes from ``$FAVEST_TUNE_CACHE``, else ``~/.cache/favest/tune.json``.  It
is rewritten atomically (temporary file, then rename), so concurrent writers never
leave a torn file; the last writer wins.  An unreadable file or entry counts as a
miss.  A shape never changes results, only speed: every shape computes the same
values.
"""
import json
import os
import tempfile


def cache_path():
    return os.environ.get("FAVEST_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "favest",
                                                               "tune.json")


def key(L, batch, precision, io_type, device_name):
    return "L%d/B%d/p%d/io%d/%s" % (int(L), int(batch), int(precision), int(io_type), device_name)


def load(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(k, shape, path=None):
    path = path or cache_path()
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    data = load(path)
    data[k] = [int(v) for v in shape]
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune-", suffix=".json")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def tune(plan, device_name=None, path=None, stream=None):
    """Give `plan` (an ``api.Plan``) its generator shape from the cache, or tune it and
    record the result.  Returns (lt, mb, nj, hit)."""
    from .api import FavestError
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    k = key(plan.L, plan.batch, plan.precision, plan.io_type, device_name)
    entry = load(path).get(k)
    if isinstance(entry, list) and len(entry) == 3:
        try:
            plan.set_gen_shape(*entry)
            return int(entry[0]), int(entry[1]), int(entry[2]), True
        except (FavestError, TypeError, ValueError):
            pass                                   # stale or edited entry: tune again
    plan.tune(stream)
    lt, mb = plan.gen_shape()
    nj = plan.gen_chains()
    store(k, (lt, mb, nj), path)
    return lt, mb, nj, False
