"""Independent NESTED HEALPix ang2pix for tests (Gorski et al. 2005, Sec. 4
of their paper): maps a direction to its pixel with a different route from
the oracle's pix2vec (ring/face location from z and phi), so that a round
trip pins the oracle."""
import math


def _spread_bits(v):
    out = 0
    for i in range(31):
        if v & (1 << i):
            out |= 1 << (2 * i)
    return out


def ang2pix_nest(level, v):
    nside = 1 << level
    x, y, z = v
    r = math.sqrt(x * x + y * y + z * z)
    z = z / r
    phi = math.atan2(y, x)
    if phi < 0:
        phi += 2 * math.pi
    za = abs(z)
    tt = phi / (math.pi / 2)  # in [0,4)
    if za <= 2.0 / 3.0:
        temp1 = nside * (0.5 + tt)
        temp2 = nside * (z * 0.75)
        jp = int(temp1 - temp2)   # ascending edge line
        jm = int(temp1 + temp2)   # descending edge line
        ifp = jp // nside
        ifm = jm // nside
        if ifp == ifm:
            face = (ifp % 4) + 4
        elif ifp < ifm:
            face = ifp % 4
        else:
            face = (ifm % 4) + 8
        ix = jm % nside
        iy = nside - (jp % nside) - 1
    else:
        ntt = min(int(tt), 3)
        tp = tt - ntt
        tmp = nside * math.sqrt(3.0 * (1.0 - za))
        jp = int(tp * tmp)
        jm = int((1.0 - tp) * tmp)
        jp = min(jp, nside - 1)
        jm = min(jm, nside - 1)
        if z >= 0:
            face = ntt
            ix = nside - jm - 1
            iy = nside - jp - 1
        else:
            face = ntt + 8
            ix = jp
            iy = jm
    return face * nside * nside + _spread_bits(ix) + 2 * _spread_bits(iy)
