"""Checkpoint and resume of a leapfrog integration (positions, velocities,
the force at the current positions, the step counter, dt, the seed, and
optionally the surrogate's coefficient ring).

The paper has no checkpointing.  Every reduction in the library sums in a
fixed order, so a run resumed from a checkpoint continues bit for bit like
the uninterrupted run; ``tests/test_checkpoint.py`` checks exactly that.

File layout (little-endian): an 8-byte magic ``ETICSCK1``, a uint32 header
length, the header (UTF-8 JSON: names, dtypes and shapes of the arrays, the
scalar state), the raw array bytes in header order, and a trailing uint32
CRC-32 of everything before it.  A file whose magic, length or checksum does
not match raises ``ValueError``.
"""
from __future__ import annotations

import json
import os
import struct
import zlib

import numpy as np
import torch

MAGIC = b"ETICSCK1"


def save(path: str, *, posm: torch.Tensor, vel: torch.Tensor, accpot: torch.Tensor, step: int,
         dt: float, seed: int = 0, extra: dict | None = None) -> None:
    """Write the state atomically (a temporary file renamed over ``path``).
    ``extra``: further named tensors (e.g. the surrogate's ring and order)."""
    arrays = {"posm": posm, "vel": vel, "accpot": accpot}
    arrays.update(extra or {})
    host = {k: v.detach().cpu().contiguous() for k, v in arrays.items()}
    header = {"step": int(step), "dt": float(dt), "seed": int(seed),
              "arrays": [{"name": k, "dtype": str(v.dtype).replace("torch.", ""),
                          "shape": list(v.shape)} for k, v in host.items()]}
    hb = json.dumps(header, sort_keys=True).encode()
    body = bytearray(MAGIC + struct.pack("<I", len(hb)) + hb)
    for v in host.values():
        body += v.view(torch.uint8).numpy().tobytes() if v.numel() else b""
    body += struct.pack("<I", zlib.crc32(bytes(body)) & 0xFFFFFFFF)
    tmp = f"{path}.tmp.{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(body)
    os.replace(tmp, path)


def load(path: str, device="cuda"):
    """Returns (arrays dict of device tensors, header dict)."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < len(MAGIC) + 8 or data[:len(MAGIC)] != MAGIC:
        raise ValueError(f"{path}: not an ETICS checkpoint")
    (crc,) = struct.unpack("<I", data[-4:])
    if zlib.crc32(data[:-4]) & 0xFFFFFFFF != crc:
        raise ValueError(f"{path}: checksum mismatch")
    (hl,) = struct.unpack("<I", data[len(MAGIC):len(MAGIC) + 4])
    o = len(MAGIC) + 4
    header = json.loads(data[o:o + hl].decode())
    o += hl
    arrays = {}
    for a in header["arrays"]:
        dt = getattr(torch, a["dtype"])
        n = int(np.prod(a["shape"])) * torch.empty(0, dtype=dt).element_size()
        buf = bytearray(data[o:o + n])
        o += n
        t = torch.frombuffer(buf, dtype=torch.uint8) if n else torch.empty(0, dtype=torch.uint8)
        arrays[a["name"]] = t.view(dt).reshape(a["shape"]).to(device)
    if o != len(data) - 4:
        raise ValueError(f"{path}: length mismatch")
    return arrays, header
