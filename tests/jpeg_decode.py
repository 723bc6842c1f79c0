"""A small baseline JPEG decoder (ITU-T T.81: sequential DCT, Huffman, 8-bit),
written for the tests from the standard and independent of both encoders.

It reads the markers the encoders write (SOI, APP0, DQT, SOF0, DHT, DRI, SOS,
RSTn, EOI), decodes the scan with restart intervals and byte stuffing,
dequantizes, applies the inverse DCT by its definition in double precision,
replicates 4:2:0 chroma, and converts JFIF YCbCr to RGB."""
from __future__ import annotations

import math

import numpy as np

ZIGZAG = [0, 1, 8, 16, 9, 2, 3, 10, 17, 24, 32, 25, 18, 11, 4, 5, 12, 19, 26, 33, 40, 48, 41, 34, 27, 20, 13, 6, 7,
          14, 21, 28, 35, 42, 49, 56, 57, 50, 43, 36, 29, 22, 15, 23, 30, 37, 44, 51, 58, 59, 52, 45, 38, 31, 39,
          46, 53, 60, 61, 54, 47, 55, 62, 63]


def _idct_matrix() -> np.ndarray:
    m = np.zeros((8, 8))
    for u in range(8):
        for x in range(8):
            m[u, x] = (1 / math.sqrt(2) if u == 0 else 1.0) * math.cos((2 * x + 1) * u * math.pi / 16) / 2
    return m


_M = _idct_matrix()


class _Bits:
    def __init__(self, data: bytes, pos: int):
        self.data, self.pos, self.acc, self.n = data, pos, 0, 0
        self.marker = None

    def _byte(self) -> int:
        if self.marker is not None:
            return 0xFF   # past a marker: feed 1s (never consumed by valid streams)
        b = self.data[self.pos]
        if b == 0xFF:
            nxt = self.data[self.pos + 1]
            if nxt == 0x00:
                self.pos += 2
                return 0xFF
            self.marker = nxt   # RSTn or EOI: stop here
            return 0xFF
        self.pos += 1
        return b

    def bit(self) -> int:
        if self.n == 0:
            self.acc, self.n = self._byte(), 8
        self.n -= 1
        return (self.acc >> self.n) & 1

    def bits(self, k: int) -> int:
        v = 0
        for _ in range(k):
            v = (v << 1) | self.bit()
        return v

    def restart(self) -> int:
        """Skip to the next marker, which must be RSTn; return n."""
        self.n = 0
        while self.marker is None:
            self._byte()
        m = self.marker
        if not (0xD0 <= m <= 0xD7):
            raise ValueError(f"expected RST marker, found FF{m:02X}")
        self.pos += 2
        self.marker = None
        return m - 0xD0


def _huff(bits, vals):
    table, code, k = {}, 0, 0
    for length in range(1, 17):
        for _ in range(bits[length - 1]):
            table[(length, code)] = vals[k]
            code += 1
            k += 1
        code <<= 1
    return table


def _decode_sym(br: _Bits, table) -> int:
    code = 0
    for length in range(1, 17):
        code = (code << 1) | br.bit()
        v = table.get((length, code))
        if v is not None:
            return v
    raise ValueError("bad Huffman code")


def _extend(v: int, s: int) -> int:
    return v - (1 << s) + 1 if s and v < (1 << (s - 1)) else v


def parse(data: bytes) -> dict:
    """Markers and tables of a baseline JFIF file (no scan decoding)."""
    if data[:2] != b"\xff\xd8" or data[-2:] != b"\xff\xd9":
        raise ValueError("missing SOI or EOI")
    pos, info = 2, {"q": {}, "h": {}, "restart": 0}
    while True:
        if data[pos] != 0xFF:
            raise ValueError("marker expected")
        m = data[pos + 1]
        length = (data[pos + 2] << 8) | data[pos + 3]
        seg = data[pos + 4:pos + 2 + length]
        if m == 0xDB:
            i = 0
            while i < len(seg):
                t = seg[i] & 15
                q = np.zeros(64, np.int32)
                for k in range(64):
                    q[ZIGZAG[k]] = seg[i + 1 + k]
                info["q"][t] = q.reshape(8, 8)
                i += 65
        elif m == 0xC0:
            info["precision"] = seg[0]
            info["height"] = (seg[1] << 8) | seg[2]
            info["width"] = (seg[3] << 8) | seg[4]
            info["comps"] = [(seg[6 + 3 * c], seg[7 + 3 * c] >> 4, seg[7 + 3 * c] & 15, seg[8 + 3 * c])
                             for c in range(seg[5])]
        elif m == 0xC4:
            i = 0
            while i < len(seg):
                cls_id = seg[i]
                bits = list(seg[i + 1:i + 17])
                n = sum(bits)
                info["h"][(cls_id >> 4, cls_id & 15)] = _huff(bits, list(seg[i + 17:i + 17 + n]))
                i += 17 + n
        elif m == 0xDD:
            info["restart"] = (seg[0] << 8) | seg[1]
        elif m == 0xDA:
            info["scan"] = [(seg[1 + 2 * c], seg[2 + 2 * c] >> 4, seg[2 + 2 * c] & 15) for c in range(seg[0])]
            info["scan_start"] = pos + 2 + length
            return info
        elif m in (0xE0,):
            pass
        else:
            raise ValueError(f"unexpected marker FF{m:02X}")
        pos += 2 + length


def decode(data: bytes) -> np.ndarray:
    """[H, W, 3] float64 RGB (not rounded) of a baseline 4:2:0 JFIF file."""
    info = parse(data)
    W, H = info["width"], info["height"]
    comps = info["comps"]
    hmax = max(c[1] for c in comps)
    vmax = max(c[2] for c in comps)
    mw, mh = -(-W // (8 * hmax)), -(-H // (8 * vmax))
    planes = {c[0]: np.zeros((mh * 8 * c[2], mw * 8 * c[1])) for c in comps}
    scan = {c[0]: (c[1], c[2]) for c in info["scan"]}
    br = _Bits(data, info["scan_start"])
    pred = {c[0]: 0 for c in comps}
    rst_expected = 0
    for mcu in range(mw * mh):
        if info["restart"] and mcu > 0 and mcu % info["restart"] == 0:
            n = br.restart()
            if n != (rst_expected & 7):
                raise ValueError("restart markers out of order")
            rst_expected += 1
            pred = {c[0]: 0 for c in comps}
        my, mx = divmod(mcu, mw)
        for cid, h, v, tq in comps:
            td, ta = scan[cid]
            for by in range(v):
                for bx in range(h):
                    zz = np.zeros(64, np.int64)
                    s = _decode_sym(br, info["h"][(0, td)])
                    pred[cid] += _extend(br.bits(s), s)
                    zz[0] = pred[cid]
                    k = 1
                    while k < 64:
                        rs = _decode_sym(br, info["h"][(1, ta)])
                        r, s = rs >> 4, rs & 15
                        if s == 0:
                            if r == 15:
                                k += 16
                                continue
                            break
                        k += r
                        zz[k] = _extend(br.bits(s), s)
                        k += 1
                    coef = np.zeros(64)
                    for kk in range(64):
                        coef[ZIGZAG[kk]] = zz[kk]
                    F = coef.reshape(8, 8) * info["q"][tq]
                    f = _M.T @ F @ _M + 128.0   # f[y, x] = sum_v sum_u M[v,y] M[u,x] F[v,u]
                    y0, x0 = (my * v + by) * 8, (mx * h + bx) * 8
                    planes[cid][y0:y0 + 8, x0:x0 + 8] = f
    Y = planes[comps[0][0]][:H, :W]
    up = []
    for cid, h, v, _ in comps[1:]:
        p = planes[cid]
        p = np.repeat(np.repeat(p, vmax // v, axis=0), hmax // h, axis=1)
        up.append(p[:H, :W])
    Cb, Cr = up[0] - 128.0, up[1] - 128.0
    return np.stack([Y + 1.402 * Cr, Y - 0.344136 * Cb - 0.714136 * Cr, Y + 1.772 * Cb], axis=-1)
