"""splitmix64 counter-based generator (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written from its published
definition.  Used only to draw synthetic inputs (indenter centres, depths,
radii, slip directions, random deformation gradients)."""

_MASK = (1 << 64) - 1


class SplitMix64:
    """Sequential splitmix64 stream seeded with an integer."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        u = (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def normal(self) -> float:
        """Standard normal via Box-Muller on two uniforms."""
        import math
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def integers(self, n: int) -> int:
        return self.next_u64() % n
