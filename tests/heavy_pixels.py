"""Check pixels where the render kernels work hardest: the rays of the tiles
whose forward walks are longest (the heaviest tiles end both render kernels),
the rays with the most evaluations among them, and every ray whose backward
walks past the forward's hit record (2048 list entries per tile)."""
import numpy as np

HIT_ENTRIES = 2048


def heavy_pixels(ws, cams, n_tiles, per_tile, seed, beyond_record=64):
    """Per camera, an [m, 2] int32 array of (column, row) pixels: per_tile rays in
    each of the n_tiles tiles with the longest forward walks over all cameras
    (half the tile's rays with the most evaluations, half at random), plus up to
    beyond_record rays whose backward walks more than HIT_ENTRIES entries.
    Returns (pixels per camera, walk lengths of the chosen tiles, rays beyond
    the record found)."""
    rng = np.random.default_rng(seed)
    ev, last, walk = ws.debug_render_state()
    tiles = np.argsort(-walk[:, 1].astype(np.int64), kind="stable")[:n_tiles]
    picks = [[] for _ in cams]
    tile0, pix0 = [], []
    t, p = 0, 0
    for c in cams:
        tile0.append(t)
        pix0.append(p)
        t += ((c.width + 15) // 16) * ((c.height + 15) // 16)
        p += c.pixels
    for tt in tiles:
        ci = int(np.searchsorted(tile0, tt, side="right") - 1)
        c = cams[ci]
        tx = (c.width + 15) // 16
        lt = int(tt) - tile0[ci]
        cx, cy = lt % tx, lt // tx
        xs, ys = np.meshgrid(np.arange(cx * 16, min(cx * 16 + 16, c.width)),
                             np.arange(cy * 16, min(cy * 16 + 16, c.height)))
        xs, ys = xs.ravel(), ys.ravel()
        rows = pix0[ci] + ys * c.width + xs
        order = np.argsort(-ev[rows, 0].astype(np.int64), kind="stable")
        k = min(per_tile, len(rows))
        top = order[: k // 2]
        rest = rng.choice(order[k // 2:], size=k - len(top), replace=False)
        for i in np.concatenate([top, rest]):
            picks[ci].append((xs[i], ys[i]))
    beyond = np.where(last > HIT_ENTRIES)[0]
    if beyond.size > beyond_record:
        beyond = rng.choice(beyond, size=beyond_record, replace=False)
    for row in beyond:
        ci = int(np.searchsorted(pix0, row, side="right") - 1)
        r = int(row) - pix0[ci]
        picks[ci].append((r % cams[ci].width, r // cams[ci].width))
    out = []
    for ci in range(len(cams)):
        arr = np.unique(np.asarray(picks[ci], np.int32).reshape(-1, 2), axis=0)
        out.append(arr)
    return out, walk[tiles, 1], int((last > HIT_ENTRIES).sum())
