"""Rendering of the instrumented build's outputs (paper Sec. 5 and Sec. 3).

- heatmap_rows(): per-byte access counts of a track buffer, reshaped into rows of a
  chosen width (the track size, a cache line, the bus width: Sec. 5 notes that the row
  width selects what the picture shows).  The device counts per 4-byte word; every leaf
  is accessed whole and aligned, so each byte of a word has the word's count.
- write_png(): grayscale or heat-coloured PNG from a 2-D count array (zlib, no imaging
  library), log-scaled.
- trace_table(): per-field read/write counts (the Trace / FieldAccessCount view).
- layout_svg(): where each leaf of the 64-byte record lands in the first bytes of a
  buffer for a layout (the layout visualisation of Sec. 3), wrapped every 64 bytes.
"""
from __future__ import annotations

import struct
import zlib

import numpy as np

LEAVES = (("x", 0, 4), ("y", 4, 4), ("z", 8, 4), ("dx", 12, 4), ("dy", 16, 4), ("dz", 20, 4),
          ("ekin", 24, 4), ("num_ia_left", 28, 4), ("id", 32, 8), ("event", 40, 4),
          ("step", 44, 4), ("slab", 48, 4), ("time", 52, 4), ("track_len", 56, 4),
          ("flags", 60, 4))


def heatmap_rows(word_counts: np.ndarray, row_bytes: int = 64, n_bytes: int | None = None):
    """Per-byte counts (each word's count repeated 4 times) reshaped to [rows, row_bytes]."""
    per_byte = np.repeat(np.asarray(word_counts, dtype=np.uint64), 4)
    if n_bytes is not None:
        per_byte = per_byte[:n_bytes]
    rows = -(-per_byte.size // row_bytes)
    out = np.zeros(rows * row_bytes, dtype=np.uint64)
    out[: per_byte.size] = per_byte
    return out.reshape(rows, row_bytes)


def used_extent(word_counts: np.ndarray) -> int:
    """Bytes up to the last accessed word."""
    nz = np.flatnonzero(np.asarray(word_counts))
    return 0 if nz.size == 0 else int(nz[-1] + 1) * 4


def _png_chunk(tag: bytes, data: bytes) -> bytes:
    return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data))


def _colour(v: np.ndarray) -> np.ndarray:
    """black -> red -> yellow -> white for v in [0, 1]."""
    r = np.clip(3 * v, 0, 1)
    g = np.clip(3 * v - 1, 0, 1)
    b = np.clip(3 * v - 2, 0, 1)
    return (np.stack([r, g, b], axis=-1) * 255).astype(np.uint8)


def write_png(path: str, counts: np.ndarray, scale: int = 1, log: bool = True) -> None:
    c = np.asarray(counts, dtype=np.float64)
    v = np.log1p(c) if log else c
    m = v.max()
    v = v / m if m > 0 else v
    img = _colour(v)
    if scale > 1:
        img = np.repeat(np.repeat(img, scale, axis=0), scale, axis=1)
    h, w, _ = img.shape
    raw = b"".join(b"\x00" + img[y].tobytes() for y in range(h))
    png = b"\x89PNG\r\n\x1a\n" + _png_chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, 8, 2, 0, 0, 0))
    png += _png_chunk(b"IDAT", zlib.compress(raw, 6)) + _png_chunk(b"IEND", b"")
    with open(path, "wb") as f:
        f.write(png)


def trace_table(trace: np.ndarray, names=("e-", "e+", "gamma")) -> str:
    """trace[3][15][2] -> a text table of reads and writes per field."""
    lines = ["field          " + "".join(f"{n + ' R':>14}{n + ' W':>14}" for n in names)]
    for f, (leaf, _, _) in enumerate(LEAVES):
        row = f"{leaf:<15}"
        for t in range(len(names)):
            row += f"{int(trace[t, f, 0]):>14}{int(trace[t, f, 1]):>14}"
        lines.append(row)
    return "\n".join(lines)


def leaf_address(layout: str, i: int, f: int, cap: int) -> int:
    """Byte address of leaf f of track i (same mapping as the device layout layer)."""
    _, off, size = LEAVES[f]
    if layout == "hotcold":  # hot 52 bytes AoSoA-32, cold fields SoA after them
        if off < 52:
            return (i // 32) * 52 * 32 + off * 32 + size * (i % 32)
        return 52 * cap + (off - 52) * cap + 4 * i
    n = {"aos": 1, "soa": cap, "aosoa8": 8, "aosoa16": 16, "aosoa32": 32, "aosoa64": 64,
         "aosoa128": 128}[layout]
    return (i // n) * 64 * n + off * n + size * (i % n)


def layout_svg(path: str, layout: str, n_tracks: int = 4, cap: int = 4, n_bytes: int = 256):
    """Boxes per (track, leaf) placed at their byte addresses, 64 bytes per row."""
    px = 10
    cols = ["#e6194b", "#3cb44b", "#ffe119", "#4363d8", "#f58231", "#911eb4", "#46f0f0",
            "#f032e6", "#bcf60c", "#fabebe", "#008080", "#e6beff", "#9a6324", "#fffac8",
            "#800000"]
    rows = n_bytes // 64
    out = [f'<svg xmlns="http://www.w3.org/2000/svg" width="{64 * px}" height="{rows * 3 * px}">']
    for i in range(n_tracks):
        for f, (leaf, _, size) in enumerate(LEAVES):
            a = leaf_address(layout, i, f, cap)
            if a >= n_bytes:
                continue
            x, y = (a % 64) * px, (a // 64) * 3 * px
            out.append(f'<rect x="{x}" y="{y}" width="{size * px}" height="{2 * px}" '
                       f'fill="{cols[f]}" stroke="black"/>')
            out.append(f'<text x="{x + 1}" y="{y + 1.4 * px}" font-size="{0.8 * px}">'
                       f'{i}:{leaf}</text>')
    out.append("</svg>")
    with open(path, "w") as fh:
        fh.write("\n".join(out))
