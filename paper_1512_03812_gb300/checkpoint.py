"""Checkpoint and resume of a batch of HMC chains (host side).

The library draws no random numbers: momenta, noise and Metropolis uniforms
come from the caller.  A chain's state between trajectories is therefore its
link angles q (FP64) plus the caller's random-generator state, and resuming
from a checkpoint reproduces the following trajectories bit for bit (the
trajectory is a deterministic function of q, p, eta and u).

File format (little-endian), one file per batch:

    8 bytes   magic  b"SMCKPT01"
    8 bytes   uint64 length H of the header
    H bytes   UTF-8 JSON header: {"chains": [[L, T], ...], "beta": [...],
              "m0": [...], "trajectory": k, "params": {...},
              "q_bytes": B, "rng_bytes": R}
    B bytes   q as float64, site-major over the chains ([N][2])
    R bytes   the random-generator state (torch.Generator.get_state()), or
              nothing
"""
from __future__ import annotations

import json
import os
import struct

import numpy as np

MAGIC = b"SMCKPT01"


def save(path, lattice, q, trajectory: int, rng_state=None, params: dict | None = None):
    """Writes the chains' link angles q ([N][2] FP64, host or device tensor),
    the index of the next trajectory, an optional generator state and
    free-form parameters (JSON-serialisable) to `path`."""
    qh = q.detach().cpu().numpy() if hasattr(q, "detach") else np.asarray(q)
    if qh.dtype != np.float64 or qh.shape != (int(lattice.N), 2):
        raise ValueError(f"q must be float64 [{lattice.N}][2], got {qh.dtype} {qh.shape}")
    qb = np.ascontiguousarray(qh).astype("<f8", copy=False).tobytes()
    rb = b"" if rng_state is None else bytes(rng_state.cpu().numpy().tobytes()
                                             if hasattr(rng_state, "cpu") else rng_state)
    header = {
        "chains": [[int(L), int(T)] for L, T in zip(lattice.L, lattice.T)],
        "beta": [float(b) for b in lattice.beta],
        "m0": [float(m) for m in lattice.m0],
        "trajectory": int(trajectory),
        "params": params or {},
        "q_bytes": len(qb),
        "rng_bytes": len(rb),
    }
    hb = json.dumps(header, sort_keys=True).encode("utf-8")
    # written beside the target, flushed to disk, then renamed over it: a
    # crash or a full disk part-way leaves the previous checkpoint intact
    tmp = os.fspath(path) + ".tmp"
    try:
        with open(tmp, "wb") as f:
            f.write(MAGIC)
            f.write(struct.pack("<Q", len(hb)))
            f.write(hb)
            f.write(qb)
            f.write(rb)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise


def load(path) -> dict:
    """Reads a checkpoint: a dict with the header's fields, "q" (numpy
    float64 [N][2]) and "rng_state" (a uint8 torch tensor for
    torch.Generator.set_state, or None)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError(f"{path}: not a checkpoint (magic {data[:8]!r})")
    (hlen,) = struct.unpack("<Q", data[8:16])
    header = json.loads(data[16:16 + hlen].decode("utf-8"))
    off = 16 + hlen
    qb = data[off:off + header["q_bytes"]]
    rb = data[off + header["q_bytes"]:off + header["q_bytes"] + header["rng_bytes"]]
    if len(qb) != header["q_bytes"] or len(rb) != header["rng_bytes"]:
        raise ValueError(f"{path}: truncated")
    out = dict(header)
    out["q"] = np.frombuffer(qb, dtype="<f8").reshape(-1, 2).copy()
    if header["rng_bytes"]:
        import torch
        out["rng_state"] = torch.frombuffer(bytearray(rb), dtype=torch.uint8)
    else:
        out["rng_state"] = None
    return out


def matches(ckpt: dict, lattice) -> bool:
    """True if the checkpoint holds chains of this lattice's shapes and
    couplings."""
    return (ckpt["chains"] == [[int(L), int(T)] for L, T in zip(lattice.L, lattice.T)]
            and np.array_equal(np.asarray(ckpt["beta"]), np.asarray(lattice.beta, dtype=float))
            and np.array_equal(np.asarray(ckpt["m0"]), np.asarray(lattice.m0, dtype=float)))
