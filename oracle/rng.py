"""SplitMix64, used as a counter-based generator (Steele, Lea & Flood, OOPSLA 2014).

The paper does not say how probe vectors are drawn beyond their distribution
(Sec. 6.2, Supp. C).  Both sides of this project draw the training probes from
the published SplitMix64 stream: output i of the stream keyed by ``key`` is
mix(key + (i + 1) * GAMMA), so any element can be drawn independently.
Python integers are used with explicit 64-bit masking.
"""
MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z):
    """The SplitMix64 output finaliser (variant 13 of Stafford's mixers)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def stream(seed, count):
    """The first ``count`` outputs of a sequential SplitMix64 generator."""
    out = []
    state = seed & MASK
    for _ in range(count):
        state = (state + GAMMA) & MASK
        out.append(mix64(state))
    return out


def at(key, i):
    """Output i (0-based) of the stream keyed by ``key``."""
    return mix64((key + (i + 1) * GAMMA) & MASK)


def probe_key(step_seed, system):
    """Stream key for the probes of one system in one training step."""
    return mix64((step_seed * 0x100000001B3 + system) & MASK)


def rademacher(step_seed, system, n, kz):
    """Rademacher probe matrix Z (n x kz) of one system, entries +-1.

    Element (i, j) takes bit 63 of output (i * kz + j) of the system's stream:
    set -> -1, clear -> +1.
    """
    key = probe_key(step_seed, system)
    z = [[0.0] * kz for _ in range(n)]
    for i in range(n):
        for j in range(kz):
            z[i][j] = -1.0 if (at(key, i * kz + j) >> 63) else 1.0
    return z


def uniform53(x):
    """A 64-bit output as a uniform in [0, 1): its top 53 bits over 2^53."""
    return (x >> 11) * (1.0 / 9007199254740992.0)


def gaussian(step_seed, system, n, kz):
    """Standard normal probe matrix Z (n x kz) of one system (Box & Muller 1958).

    Element (i, j) takes outputs 2e and 2e + 1 (e = i * kz + j) of the system's
    stream as uniforms u1, u2 and returns sqrt(-2 ln(1 - u1)) cos(2 pi u2); 1 - u1
    is never 0.
    """
    import math
    key = probe_key(step_seed, system)
    z = [[0.0] * kz for _ in range(n)]
    for i in range(n):
        for j in range(kz):
            e = i * kz + j
            u1 = uniform53(at(key, 2 * e))
            u2 = uniform53(at(key, 2 * e + 1))
            z[i][j] = math.sqrt(-2.0 * math.log1p(-u1)) * math.cos(2.0 * math.pi * u2)
    return z
