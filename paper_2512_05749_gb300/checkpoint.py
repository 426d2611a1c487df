"""Checkpoint and resume of the WSSR optimiser state.

The library keeps nothing between steps: the state a run carries from one
step to the next is the subspace V (M x r FP32), its Ritz values sigma (r
FP64), the step index, the counters of the caller's random streams, and for
the history-averaged step (Section 4.1) L-bar (r FP64). Because every
reduction in the library runs in a fixed order, a run resumed from a
checkpoint repeats the uninterrupted run bit for bit.

File format (all little-endian):
  8 bytes   magic b"WSSRCKPT"
  u32       version (1)
  u32       flags (bit 0: L-bar present)
  i64       M, i64 r, i64 step, u64 rng_counter
  M*r f32   V, row-major
  r   f64   sigma
  r   f64   L-bar (if flag bit 0)
  u64       CRC-32 (zlib) of every byte above
"""
import os
import struct
import zlib

import numpy as np

MAGIC = b"WSSRCKPT"
VERSION = 1
_HEAD = struct.Struct("<8sIIqqqQ")


class CheckpointError(ValueError):
    pass


def _digest(parts) -> int:
    """CRC-32 (zlib) of the header and the arrays' bytes, in file order."""
    c = 0
    for p in parts:
        c = zlib.crc32(p if isinstance(p, (bytes, bytearray, memoryview)) else memoryview(p).cast("B"), c)
    return c


def _to_numpy(t, dtype):
    try:
        import torch
        if isinstance(t, torch.Tensor):
            t = t.detach().to("cpu").numpy()
    except ImportError:
        pass
    return np.ascontiguousarray(np.asarray(t), dtype=dtype)


def save(path: str, step: int, V, sigma, Lbar=None, rng_counter: int = 0) -> None:
    """Write the state atomically (to path + ".tmp", then rename)."""
    Vn = _to_numpy(V, "<f4")
    if Vn.ndim != 2:
        raise CheckpointError("V must be M x r")
    M, r = Vn.shape
    sn = _to_numpy(sigma, "<f8").reshape(-1)
    if sn.shape[0] != r:
        raise CheckpointError("sigma must have r entries")
    ln = None if Lbar is None else _to_numpy(Lbar, "<f8").reshape(-1)
    if ln is not None and ln.shape[0] != r:
        raise CheckpointError("L-bar must have r entries")
    head = _HEAD.pack(MAGIC, VERSION, 1 if ln is not None else 0, M, r, int(step), int(rng_counter))
    parts = [head, Vn, sn] + ([ln] if ln is not None else [])
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(head)
        for a in parts[1:]:
            f.write(a.tobytes())
        f.write(struct.pack("<Q", _digest(parts)))
    os.replace(tmp, path)


def load(path: str, device=None):
    """Read a checkpoint: returns dict(step, rng_counter, V, sigma, Lbar or None).
    With a device, V / sigma / L-bar come back as torch tensors on it."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < _HEAD.size + 8:
        raise CheckpointError("file too short")
    magic, version, flags, M, r, step, rng = _HEAD.unpack_from(data, 0)
    if magic != MAGIC:
        raise CheckpointError("not a WSSR checkpoint")
    if version != VERSION:
        raise CheckpointError(f"unsupported checkpoint version {version}")
    if M < 1 or r < 1:
        raise CheckpointError("bad shape in header")
    has_l = bool(flags & 1)
    need = _HEAD.size + 4 * M * r + 8 * r + (8 * r if has_l else 0) + 8
    if len(data) != need:
        raise CheckpointError(f"size {len(data)} does not match the header ({need})")
    o = _HEAD.size
    V = np.frombuffer(data, dtype="<f4", count=M * r, offset=o).reshape(M, r).copy()
    o += 4 * M * r
    sigma = np.frombuffer(data, dtype="<f8", count=r, offset=o).copy()
    o += 8 * r
    Lbar = None
    if has_l:
        Lbar = np.frombuffer(data, dtype="<f8", count=r, offset=o).copy()
        o += 8 * r
    (h,) = struct.unpack_from("<Q", data, o)
    parts = [data[:_HEAD.size], V, sigma] + ([Lbar] if has_l else [])
    if h != _digest(parts):
        raise CheckpointError("checksum mismatch")
    out = {"step": step, "rng_counter": rng, "V": V, "sigma": sigma, "Lbar": Lbar}
    if device is not None:
        import torch
        out["V"] = torch.from_numpy(V).to(device)
        out["sigma"] = torch.from_numpy(sigma).to(device)
        if Lbar is not None:
            out["Lbar"] = torch.from_numpy(Lbar).to(device)
    return out
