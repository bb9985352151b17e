"""Host-side partition function Q(T), passed to the library as a scalar per temperature.

pyROX reads tabulated partition functions from the line-list databases ("Download and
read files"); a table of Q at integer temperatures is interpolated linearly, and a
closed form a*T^1.5 (the rigid-rotor high-temperature limit of a non-linear molecule)
serves workloads that define one.
"""
import bisect


class PartitionFunction:
    def __init__(self, spec):
        """spec: ('analytic', a) for Q = a*T^1.5, or ('table', T_K, Q) with ascending T_K."""
        self.kind = spec[0]
        if self.kind == "analytic":
            self.a = float(spec[1])
        elif self.kind == "table":
            self.t = [float(v) for v in spec[1]]
            self.q = [float(v) for v in spec[2]]
        else:
            raise ValueError("unknown partition-function spec %r" % (spec[0],))

    def __call__(self, T):
        T = float(T)
        if self.kind == "analytic":
            return self.a * T ** 1.5
        if T < self.t[0] or T > self.t[-1]:
            raise ValueError("T = %g K outside the partition-function table" % T)
        k = bisect.bisect_right(self.t, T) - 1
        if k >= len(self.t) - 1:
            return self.q[-1]
        w = (T - self.t[k]) / (self.t[k + 1] - self.t[k])
        return (1.0 - w) * self.q[k] + w * self.q[k + 1]
