"""Checkpoints and step logs of DNN-MG runs (host-side file I/O only).

A checkpoint holds the solution state of a context (FP64, its solved
level), the network's FP32 parameters, the feature statistics of its inputs
and the configuration, so that a run (a spin-up, a trained network) can be
resumed in a new process.  The network's recurrent memory is not part of it:
after `load` it restarts at zero, as after any `set_state`.

File format, all numbers little-endian:

    8 bytes    magic b"DNNMGCK1"
    4 bytes    uint32, length H of the header
    H bytes    UTF-8 JSON: {"meta": {...}, "arrays": [{"name", "dtype", "shape",
               "offset", "nbytes"}, ...]}
    blobs      each array's raw bytes at its offset from the end of the header,
               every offset a multiple of 16

A step log is a JSON-lines file with one object per time step (the step
statistics of `Context.step` plus whatever the caller adds).
"""
import json
import struct

import numpy as np

MAGIC = b"DNNMGCK1"
_ALIGN = 16
_DTYPES = ("<f8", "<f4", "<u2", "<i4", "<i8")

# configuration fields that define the discrete problem and the network: a
# checkpoint only loads into a context that agrees on all of them
PROBLEM_KEYS = ("level_solve", "level_coarse", "replaced_levels", "obstacle_i0", "obstacle_j0",
                "hidden", "gru_layers", "mlp_width", "lps_mode")


def write(path, arrays, meta=None):
    """Write named numpy arrays (float64/float32/uint16/int32/int64) and a
    JSON-serialisable meta dict."""
    entries, blobs, off = [], [], 0
    for name, a in arrays.items():
        a = np.ascontiguousarray(a)
        dt = a.dtype.newbyteorder("<").str
        if dt not in _DTYPES:
            raise ValueError(f"array {name}: unsupported dtype {a.dtype}")
        raw = a.astype(dt, copy=False).tobytes()
        entries.append({"name": name, "dtype": dt, "shape": list(a.shape), "offset": off,
                        "nbytes": len(raw)})
        pad = (-len(raw)) % _ALIGN
        blobs.append(raw + b"\0" * pad)
        off += len(raw) + pad
    header = json.dumps({"meta": meta or {}, "arrays": entries}).encode("utf-8")
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(header)))
        f.write(header)
        for b in blobs:
            f.write(b)


def read(path):
    """(meta, {name: array}) of a checkpoint file; ValueError if it is not one
    or is truncated."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC or len(data) < 12:
        raise ValueError(f"{path}: not a DNN-MG checkpoint")
    (hlen,) = struct.unpack("<I", data[8:12])
    if 12 + hlen > len(data):
        raise ValueError(f"{path}: truncated header")
    head = json.loads(data[12:12 + hlen].decode("utf-8"))
    base = 12 + hlen
    arrays = {}
    for e in head["arrays"]:
        lo, hi = base + e["offset"], base + e["offset"] + e["nbytes"]
        if e["dtype"] not in _DTYPES or hi > len(data):
            raise ValueError(f"{path}: bad entry {e['name']}")
        arrays[e["name"]] = np.frombuffer(data[lo:hi], dtype=e["dtype"]).reshape(e["shape"]).copy()
    return head["meta"], arrays


def _config_dict(cfg):
    return {k: getattr(cfg, k) for k, _ in cfg._fields_}


def save(ctx, path, feature_stats=None, meta=None):
    """Checkpoint of a Context: state, network parameters (when the context
    has a network of a supported size), the given feature statistics
    (mean, std) and the configuration; `meta` is stored alongside."""
    from . import dnnmg
    arrays = {"state": ctx.get_state().cpu().numpy()}
    try:
        arrays["weights"] = ctx.get_weights().numpy()
    except dnnmg.DnnmgError:
        pass  # no network of a supported size
    if feature_stats is not None:
        mean, std = feature_stats
        arrays["feat_mean"] = np.asarray(mean, dtype=np.float32)
        arrays["feat_std"] = np.asarray(std, dtype=np.float32)
    write(path, arrays, {"config": _config_dict(ctx.cfg), **(meta or {})})


def load(ctx, path):
    """Restore a checkpoint into a Context whose problem-defining
    configuration fields agree with the saved ones; returns the stored meta.
    ValueError on a mismatch."""
    import torch
    meta, arrays = read(path)
    saved, now = meta.get("config", {}), _config_dict(ctx.cfg)
    bad = [k for k in PROBLEM_KEYS if k in saved and saved[k] != now[k]]
    if bad:
        raise ValueError("checkpoint was written for another problem: " +
                         ", ".join(f"{k}={saved[k]} (context {now[k]})" for k in bad))
    x = arrays["state"]
    if x.shape != (ctx.ndof(ctx.cfg.level_solve),):
        raise ValueError(f"state of {x.shape[0]} unknowns, context has "
                         f"{ctx.ndof(ctx.cfg.level_solve)}")
    ctx.set_state(torch.from_numpy(x).cuda())
    if "weights" in arrays:
        ctx.set_weights(arrays["weights"])
    if "feat_mean" in arrays:
        ctx.set_feature_stats(arrays["feat_mean"], arrays["feat_std"])
    return meta


class StepLog:
    """Append-only JSON-lines log of time steps."""

    def __init__(self, path):
        self._f = open(path, "a", encoding="utf-8")

    def write(self, step, stats, **extra):
        self._f.write(json.dumps({"step": step, **stats, **extra}) + "\n")
        self._f.flush()

    def close(self):
        self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_log(path):
    with open(path, encoding="utf-8") as f:
        return [json.loads(line) for line in f if line.strip()]
