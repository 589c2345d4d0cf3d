"""Counter-based normal deviates for the moving goals (tracking task).

The 64-bit finaliser of SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) hashes a key built from
(seed, env, chain, step); two hashed words give four 24-bit uniforms in
(0, 1) and the Box-Muller transform gives normal deviates.  Integer
arithmetic is exact (numpy uint64 wraps modulo 2^64), so both sides of a
parity test draw identical uniforms.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_next(state):
    """One SplitMix64 step: (new state, output)."""
    with np.errstate(over="ignore"):
        s = np.uint64(state) + GOLDEN
    return s, mix64(s)


def _key_words(seed, env, lo, step, shift):
    u64 = lambda x: np.asarray(x).astype(np.uint64)
    with np.errstate(over="ignore"):
        key = mix64(u64(seed) + GOLDEN)
        key = mix64(key + GOLDEN + u64(env))
        key = mix64(key + GOLDEN + ((u64(step) << np.uint64(shift)) | u64(lo)))
        return mix64(key + GOLDEN), mix64(key + GOLDEN + GOLDEN)


def _box_muller(w0, w1):
    s = 2.0 ** -24
    top = lambda w: ((w >> np.uint64(40)).astype(np.float64) + 0.5) * s
    mid = lambda w: (((w >> np.uint64(16)) & np.uint64(0xFFFFFF)).astype(np.float64) + 0.5) * s
    u0, u1, u2, u3 = top(w0), mid(w0), top(w1), mid(w1)
    r0 = np.sqrt(-2.0 * np.log(u0))
    r1 = np.sqrt(-2.0 * np.log(u2))
    return np.stack([r0 * np.cos(2 * np.pi * u1), r0 * np.sin(2 * np.pi * u1),
                     r1 * np.cos(2 * np.pi * u3), r1 * np.sin(2 * np.pi * u3)], -1)


def action_noise(seed, env, block, step):
    """Four standard normal deviates for (seed, env, joint block, step) of
    the policy's exploration noise: joint j of an env uses block j // 4,
    component j % 4 (key: step << 5 | block).  Returns [..., 4] float64."""
    w0, w1 = _key_words(seed, env, block, step, 5)
    return _box_muller(w0, w1)


def goal_noise(seed, env, chain, step):
    """Three standard normal deviates for (seed, env, chain, step); array
    arguments broadcast.  Returns [..., 3] float64."""
    u64 = lambda x: np.asarray(x).astype(np.uint64)
    with np.errstate(over="ignore"):
        key = mix64(u64(seed) + GOLDEN)
        key = mix64(key + GOLDEN + u64(env))
        key = mix64(key + GOLDEN + ((u64(step) << np.uint64(2)) | u64(chain)))
        w0 = mix64(key + GOLDEN)
        w1 = mix64(key + GOLDEN + GOLDEN)
    s = 2.0 ** -24
    top = lambda w: ((w >> np.uint64(40)).astype(np.float64) + 0.5) * s
    mid = lambda w: (((w >> np.uint64(16)) & np.uint64(0xFFFFFF)).astype(np.float64) + 0.5) * s
    u0, u1, u2, u3 = top(w0), mid(w0), top(w1), mid(w1)
    r0 = np.sqrt(-2.0 * np.log(u0))
    r1 = np.sqrt(-2.0 * np.log(u2))
    return np.stack([r0 * np.cos(2 * np.pi * u1), r0 * np.sin(2 * np.pi * u1),
                     r1 * np.cos(2 * np.pi * u3)], -1)
