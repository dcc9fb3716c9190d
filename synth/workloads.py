"""Plain-data description of the synthetic workloads (no method arithmetic).

Every number here is either a constant of a workload recipe or drawn from a
SplitMix64 stream (gen.py).  Dtype codes match the library's: f32=0, f64=1,
i32=2, bf16=3.  A section lists the op it runs, its operand field ids, the
fields it reads at record i (read), writes at record i (write) and reads at
record perm[i] (read_at_perm), and its fp32 constants (params).
"""
from dataclasses import dataclass, field as dc_field
from typing import List, Tuple

import numpy as np

from . import gen

F32, F64, I32, BF16 = 0, 1, 2, 3
DTYPE_SIZE = {F32: 4, F64: 8, I32: 4, BF16: 2}
DTYPE_NP = {F32: np.float32, F64: np.float64, I32: np.int32, BF16: np.uint16}
DTYPE_NAME = {F32: "f32", F64: "f64", I32: "i32", BF16: "bf16"}

# Section op names; the numeric codes are the library's adha_op values.
OPS = dict(madd3=1, xorshift=2, add=3, mix=4, drift=5, bin=6, ke=7, flags=8, gather=9, kick=10,
           axpb=11, mul=12, tanh=13, assign=14, reduce=15)

DT = 2.0 ** -7           # time step of the particle sections (a power of two: dt*v is exact)


@dataclass(frozen=True)
class Field:
    name: str
    dtype: int
    kind: str            # synth value recipe (gen.KIND)


@dataclass(frozen=True)
class Section:
    op: str
    args: Tuple[int, ...] = ()
    read: frozenset = frozenset()
    write: frozenset = frozenset()
    read_at_perm: frozenset = frozenset()
    params: Tuple[float, ...] = ()
    table: Tuple[float, ...] = ()        # constants beyond params (assign: K x d centroids)

    @property
    def touched(self):
        return self.read | self.write | self.read_at_perm


@dataclass
class Workload:
    name: str
    n: int
    fields: List[Field]
    seed: int
    sections: List[Section]
    candidates: str = "ads"          # "ads": ODS candidates + AoS + SoA; "aos_soa": AoS and SoA only
    loss_weights: Tuple[float, ...] = ()
    has_perm: bool = False
    extra: dict = dc_field(default_factory=dict)

    @property
    def F(self):
        return len(self.fields)

    @property
    def dtypes(self):
        return [f.dtype for f in self.fields]

    def field_key(self, f):
        return gen.key(self.seed, f)

    def perm_key(self):
        return gen.key(self.seed, 1000)

    def values(self, f, idx=None, n=None, i0=0):
        """Initial values of field f for records idx (or i0..i0+n)."""
        if idx is None and n is None:
            n = self.n
        return gen.fill(self.fields[f].kind, self.field_key(f), n=n, i0=i0, idx=idx)

    def perm(self):
        return gen.perm_i32(self.perm_key(), self.n)

    def with_n(self, n):
        w = Workload(self.name, n, self.fields, self.seed, self.sections, self.candidates,
                     self.loss_weights, self.has_perm, dict(self.extra))
        return w


def _fs(*xs):
    return frozenset(xs)


def config1(n=65536):
    """6 fields (f0..f3 fp32 U[-1,1), i0,i1 int32 U[0,2^20)), 3 sections, AoS/SoA candidates only."""
    flds = [Field("f0", F32, "F32_PM1"), Field("f1", F32, "F32_PM1"), Field("f2", F32, "F32_PM1"),
            Field("f3", F32, "F32_PM1"), Field("i0", I32, "I32_U20"), Field("i1", I32, "I32_U20")]
    secs = [Section("madd3", (0, 1, 2), _fs(0, 1, 2), _fs(2)),          # f2 = f0*f1 + f2
            Section("xorshift", (4, 5), _fs(3, 4), _fs(5)),            # i1 = i0 ^ (i0>>3); f3 read too
            Section("add", (0, 3, 0), _fs(0, 1, 2, 3, 4, 5), _fs(0))]  # f0 = f0 + f3; reads every field
    return Workload("config1_tiny_n65536", n, flds, 0, secs, candidates="aos_soa")


def _bernoulli_sections(seed, F, n_rand, p):
    kr, kw = gen.key(seed, 2000), gen.key(seed, 2001)
    secs = []
    for s in range(n_rand):
        r = {f for f in range(F) if gen.unit(kr, s * F + f) < p}
        w = {f for f in range(F) if gen.unit(kw, s * F + f) < p}
        if not w:
            w = {min(r)} if r else {0}
        r |= w                                   # every write is a read-modify-write
        secs.append(Section("mix", (), frozenset(r), frozenset(w)))
    secs.append(Section("mix", (), frozenset(range(F)), frozenset(range(F))))
    return secs


def config2(n=1 << 24):
    """16 fields (8 fp32, 4 fp64, 4 int32 = 80 B AoS), 8 Bernoulli(0.3) sections + 1 all-field section."""
    flds = ([Field("a%d" % k, F32, "F32_PM1") for k in range(8)]
            + [Field("d%d" % k, F64, "F64_PM1") for k in range(4)]
            + [Field("i%d" % k, I32, "I32_U20") for k in range(4)])
    return Workload("config2_layout_stress_n%d" % n, n, flds, 1, _bernoulli_sections(1, 16, 8, 0.3))


def config3(n=1 << 25):
    """Particles: 12 fields (52 B data, 56 B AoS), 10 sections incl. a gather through a permutation."""
    flds = [Field("px", F32, "F32_01"), Field("py", F32, "F32_01"), Field("pz", F32, "F32_01"),
            Field("vx", F32, "F32_NORMAL"), Field("vy", F32, "F32_NORMAL"), Field("vz", F32, "F32_NORMAL"),
            Field("mass", F32, "F32_LOGNORMAL"), Field("charge", F32, "F32_SIGN"),
            Field("id", I32, "I32_IOTA"), Field("cell", I32, "ZERO32"), Field("flags", I32, "ZERO32"),
            Field("energy", F64, "ZERO64")]
    PX, PY, PZ, VX, VY, VZ, M, Q, ID, CELL, FL, E = range(12)
    drift = Section("drift", (PX, PY, PZ, VX, VY, VZ), _fs(PX, PY, PZ, VX, VY, VZ), _fs(PX, PY, PZ), params=(DT,))
    binning = Section("bin", (PX, PY, PZ, CELL), _fs(PX, PY, PZ), _fs(CELL), params=(128.0,))
    ke = Section("ke", (VX, VY, VZ, M, E), _fs(VX, VY, VZ, M), _fs(E))
    flags = Section("flags", (FL, E), _fs(FL, E), _fs(FL), params=(1.5,))
    gather = Section("gather", (VX, VY, VZ, PX, PY, PZ, Q), _fs(VX, VY, VZ), _fs(VX, VY, VZ),
                     _fs(PX, PY, PZ, Q), params=(DT,))
    kick = Section("kick", (VX, VY, VZ, Q), _fs(VX, VY, VZ, Q), _fs(VX, VY, VZ),
                   params=(DT, 0.125, -0.0625, 0.03125))
    secs = [drift, binning, ke, flags, gather, kick, drift, binning, ke, flags]
    return Workload("config3_particles_n%d" % n, n, flds, 2, secs, has_perm=True)


def config5(n=1 << 26, n_sections=64):
    """24 fp32 N(0,1) fields, 64 drawn sections (a*x+b, x*y, tanh x), linear loss sum_f c_f sum_i field_f."""
    F = 24
    flds = [Field("x%d" % k, F32, "F32_NORMAL") for k in range(F)]
    seed = 4
    secs = []
    for s in range(n_sections):
        k = gen.key(seed, 3000 + s)
        u = gen.unit(k, 0)
        x, y, z = (int(gen.unit(k, j) * F) for j in (1, 2, 3))
        if u < 0.4:
            a = float(np.float32(2.0 * gen.unit(k, 4) - 1.0))
            b = float(np.float32(2.0 * gen.unit(k, 5) - 1.0))
            secs.append(Section("axpb", (x, z), _fs(x), _fs(z), params=(a, b)))
        elif u < 0.7:
            secs.append(Section("mul", (x, y, z), _fs(x, y), _fs(z)))
        else:
            secs.append(Section("tanh", (x, z), _fs(x), _fs(z)))
    kc = gen.key(seed, 2999)
    c = tuple(float(np.float32(2.0 * gen.unit(kc, f) - 1.0)) for f in range(F))
    return Workload("config5_differentiable_n%d" % n, n, flds, seed, secs, loss_weights=c)


def kmeans(n=8388608, n_features=32, k=5, seed=6):
    """K-Means-shaped program (the paper's second benchmark, Table 1: 8388608 inputs, 32 fields,
    2 sections): 32 fp32 features U[-1,1) and an int32 membership field (zero at start);
    section 1 assigns every record to its nearest of k seeded centroids (U[-1,1) fp32),
    section 2 reduces every feature into per-cluster fixed-point sums and counts."""
    flds = [Field("x%d" % j, F32, "F32_PM1") for j in range(n_features)] + [Field("member", I32, "ZERO32")]
    M = n_features
    feats = frozenset(range(n_features))
    kc = gen.key(seed, 5000)
    cent = tuple(float(np.float32(2.0 * gen.unit(kc, i) - 1.0)) for i in range(k * n_features))
    assign = Section("assign", (M, k), feats, _fs(M), table=cent)
    reduce = Section("reduce", (M, k), feats | _fs(M), frozenset())
    return Workload("kmeans_n%d_f%d_k%d" % (n, n_features, k), n, flds, seed, [assign, reduce])


def medical(n=256 ** 3, seed=7):
    """Medical-image-registration-shaped program (the paper's first benchmark, Table 1 and Table 2:
    a 256^3 volume, 7 sections over the fields V1..V3, U1..U3, S, T, interpT).  Sections 1-3 move
    the vector fields together (a gather of T and U at a displaced record, a kick by S, a drift of
    U by V), sections 4-7 are elementwise updates of the scalar fields.  Values: V N(0,1), U U[0,1),
    S, T and interpT U[-1,1); the displaced record is a seeded random permutation."""
    flds = [Field("V1", F32, "F32_NORMAL"), Field("V2", F32, "F32_NORMAL"), Field("V3", F32, "F32_NORMAL"),
            Field("U1", F32, "F32_01"), Field("U2", F32, "F32_01"), Field("U3", F32, "F32_01"),
            Field("S", F32, "F32_PM1"), Field("T", F32, "F32_PM1"), Field("interpT", F32, "F32_PM1")]
    V1, V2, V3, U1, U2, U3, S, T, IT = range(9)
    gather = Section("gather", (V1, V2, V3, U1, U2, U3, T), _fs(V1, V2, V3), _fs(V1, V2, V3),
                     _fs(U1, U2, U3, T), params=(DT,))
    kick = Section("kick", (V1, V2, V3, S), _fs(V1, V2, V3, S), _fs(V1, V2, V3), params=(DT, 0.25, -0.125, 0.0625))
    drift = Section("drift", (U1, U2, U3, V1, V2, V3), _fs(U1, U2, U3, V1, V2, V3), _fs(U1, U2, U3), params=(DT,))
    interp = Section("axpb", (T, IT), _fs(T), _fs(IT), params=(0.75, 0.125))
    scale = Section("mul", (T, IT, S), _fs(T, IT), _fs(S))
    update = Section("madd3", (U1, V1, T), _fs(U1, V1, T), _fs(T))
    squash = Section("tanh", (S, IT), _fs(S), _fs(IT))
    secs = [gather, kick, drift, interp, scale, update, squash]
    return Workload("medical_n%d" % n, n, flds, seed, secs, has_perm=True)


def config4_arrays(seed=3, n_arrays=256, n_scale=1.0):
    """256 record arrays: N log-uniform in [2^10, 2^22), F uniform in [4,32], dtypes uniform per field,
    source AoS in declared order, target a random set partition (shuffle, cut into groups of 1..8).
    Returns a list of dicts with keys n, dtypes, src (list of groups), dst (list of groups), keys."""
    arrays = []
    for a in range(n_arrays):
        k = gen.key(seed, 4000 + a)
        n = int(2.0 ** (10.0 + 12.0 * gen.unit(k, 0)))
        n = max(1, int(n * n_scale))
        F = 4 + int(gen.unit(k, 1) * 29)
        dtypes = [int(gen.unit(k, 2 + f) * 4) for f in range(F)]
        order = list(range(F))
        ks = gen.key(seed, 6000 + a)
        for i in range(F - 1, 0, -1):                      # Fisher-Yates
            j = int(gen.unit(ks, F - 1 - i) * (i + 1))
            order[i], order[j] = order[j], order[i]
        dst, pos, g = [], 0, 0
        while pos < F:
            size = 1 + int(gen.unit(ks, 100 + g) * 8)
            dst.append(order[pos:pos + size])
            pos += size
            g += 1
        kinds = {F32: "RAW32", F64: "RAW64", I32: "RAW32", BF16: "RAW16"}
        arrays.append(dict(n=n, dtypes=dtypes, src=[list(range(F))], dst=dst,
                           kinds=[kinds[d] for d in dtypes],
                           keys=[gen.key(seed, 100000 + a * 64 + f) for f in range(F)]))
    return arrays


def tiny_workload(seed, F_max=8, n=37, n_sections=4):
    """A random small mixed-dtype workload of 'mix' sections, for fuzz tests on both sides."""
    k = gen.key(seed, 7000)
    F = 2 + int(gen.unit(k, 0) * (F_max - 1))
    kinds = {F32: "F32_PM1", F64: "F64_PM1", I32: "I32_U20", BF16: "RAW16"}
    dts = [int(gen.unit(k, 1 + f) * 3) for f in range(F)]
    flds = [Field("t%d" % f, d, kinds[d]) for f, d in enumerate(dts)]
    secs = _bernoulli_sections(seed, F, n_sections, 0.4)
    return Workload("tiny_seed%d" % seed, n, flds, seed, secs)


def workload(name, **kw):
    return {"config1": config1, "config2": config2, "config3": config3, "config5": config5, "kmeans": kmeans,
            "medical": medical}[name](**kw)
