"""Variant-space definition and code generation for the SIMT SGEMM family.

The variant space is the Cartesian grid of tuning parameters

    CTA tile BM, BN in {32, 64, 128, 256}     K-step BK in {8, 16, 32}
    thread tile TM x TN in {4, 8}^2            in-warp k-groups KL in {1, 2, 4}
    vector width VEC in {1, 2, 4}              pipeline depth STAGES in {2, 3, 4}
    cluster split-K SPLITK in {1, 2, 4, 8}     staging: cp.async with M-major A,
                                               cp.async with K-major A, TMA with K-major A
    FMA form F2 in {0: fmaf, 1: packed fma.rn.f32x2}

pruned by static validity rules (threads per CTA in {64, 128, 256, 512},
lane layout that tiles the warp, BK a multiple of 4*KL, shared memory within
227 KB, the split-K reduction tile within shared memory, rows divisible by
SPLITK, register tile at most 64 accumulators).  Like the paper's dataset
(a hand-tuned subset followed by a random selection from the kernel space,
Section V-D), the compiled family is a fixed core of conventional
configurations plus a SplitMix64-seeded stratified sample of the rest, about
380 variants in total.  Output: ``variant_table.inc`` (every variant as an
X-macro row) and ``variants_XX.cu`` translation units that instantiate them,
compiled in parallel.
"""

from __future__ import annotations

import itertools
import math
import os
import sys

TARGET_COUNT = 384
SAMPLE_SEED = 20250715
N_TUS = 24
SMEM_LIMIT = 232448

FAMILIES = {  # name -> (LOADER, AKM)
    "cpm": (0, 0),
    "cpk": (0, 1),
    "tmk": (1, 1),
}


def _mix(z):
    m = (1 << 64) - 1
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & m
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & m
    return z ^ (z >> 31)


def _rand(seed, i):
    return _mix((seed + (i + 1) * 0x9E3779B97F4A7C15) & ((1 << 64) - 1))


def round_up(x, m):
    return (x + m - 1) // m * m


def lane_layout(BM, BN, TM, TN, KL):
    """(LM, LN) for a warp: LM*LN = 32/KL, warp tile as square as possible."""
    lanes = 32 // KL
    best = None
    for lm in (1, 2, 4, 8, 16, 32):
        if lanes % lm:
            continue
        ln = lanes // lm
        wm, wn = lm * TM, ln * TN
        if wm > BM or wn > BN or BM % wm or BN % wn:
            continue
        score = (abs(math.log2(wm / wn)), -wn)
        if best is None or score < best[0]:
            best = (score, lm, ln)
    return None if best is None else (best[1], best[2])


def smem_bytes(BM, BN, BK, STAGES, SPLITK, LOADER, AKM):
    pad = 4 if LOADER == 0 else 0
    a_stage = round_up(BM * BK * 4 if AKM else BK * (BM + pad) * 4, 1024)
    b_stage = round_up(BK * (BN + pad) * 4, 1024)
    pipe = STAGES * (a_stage + b_stage)
    red = BM * (BN + 4) * 4 if SPLITK > 1 else 0
    bars = 16 * STAGES if LOADER == 1 else 0
    return max(pipe, red) + bars + 1024


def name_of(v):
    return ("s{BM}x{BN}x{BK}_w{WM}x{WN}_t{TM}x{TN}_kl{KL}_v{VEC}_p{STAGES}_sk{SPLITK}_{fam}"
            .format(**v)) + ("_ffma2" if v.get("F2") else "")


def enumerate_space():
    out = []
    for BM, BN in itertools.product((32, 64, 128, 256), repeat=2):
        for TM, TN in itertools.product((4, 8), repeat=2):
            for KL in (1, 2, 4):
                threads = BM * BN * KL // (TM * TN)
                if threads not in (64, 128, 256, 512) or TM % KL:
                    continue
                lay = lane_layout(BM, BN, TM, TN, KL)
                if lay is None:
                    continue
                LM, LN = lay
                WM, WN = LM * TM, LN * TN
                for BK in (8, 16, 32):
                    if BK % (4 * KL):
                        continue
                    for fam, (LOADER, AKM) in FAMILIES.items():
                        for VEC in (1, 2, 4):
                            for STAGES in (2, 3, 4):
                                for SPLITK in (1, 2, 4, 8):
                                    if BM % SPLITK:
                                        continue
                                    sm = smem_bytes(BM, BN, BK, STAGES, SPLITK, LOADER, AKM)
                                    if sm > SMEM_LIMIT:
                                        continue
                                    for F2 in (0, 1):
                                        v = dict(BM=BM, BN=BN, BK=BK, WM=WM, WN=WN, TM=TM, TN=TN, KL=KL,
                                                 VEC=VEC, STAGES=STAGES, SPLITK=SPLITK, LOADER=LOADER, AKM=AKM,
                                                 F2=F2, fam=fam, threads=threads, smem=sm)
                                        v["name"] = name_of(v)
                                        out.append(v)
    return out


def core_set(space):
    """Conventional configurations (the hand-picked part of the family)."""
    by_name = {v["name"]: v for v in space}
    want = []
    tiles = [  # BM, BN, TM, TN, KL
        (128, 128, 8, 8, 1), (128, 256, 8, 8, 1), (256, 128, 8, 8, 1), (128, 64, 8, 8, 1),
        (64, 128, 8, 8, 1), (64, 64, 8, 8, 1), (64, 64, 4, 4, 1), (64, 64, 4, 8, 2), (32, 64, 4, 4, 1),
        (32, 32, 4, 4, 2), (64, 32, 4, 4, 1),
    ]
    for BM, BN, TM, TN, KL in tiles:
        lay = lane_layout(BM, BN, TM, TN, KL)
        if lay is None:
            continue
        WM, WN = lay[0] * TM, lay[1] * TN
        for fam in FAMILIES:
            for BK in (8, 16):
                for STAGES in (2, 3, 4):
                    for SPLITK in (1, 4) if BM * BN <= 128 * 128 else (1,):
                        for F2 in (0, 1):
                            v = dict(BM=BM, BN=BN, BK=BK, WM=WM, WN=WN, TM=TM, TN=TN, KL=KL, VEC=4,
                                     STAGES=STAGES, SPLITK=SPLITK, fam=fam, F2=F2)
                            n = name_of(v)
                            if n in by_name and (STAGES == 3 or SPLITK == 1 and BK == 8):
                                want.append(n)
    seen, out = set(), []
    for n in want:
        if n not in seen:
            seen.add(n)
            out.append(by_name[n])
    return out


def stratified_sample(space, exclude, count, seed):
    """Seeded sample spread over (tile, split-K, family) strata."""
    strata = {}
    for v in space:
        if v["name"] in exclude:
            continue
        strata.setdefault((v["BM"], v["BN"], v["SPLITK"], v["fam"]), []).append(v)
    keys = sorted(strata)
    for k in keys:  # deterministic shuffle of each stratum
        lst = strata[k]
        for i in range(len(lst) - 1, 0, -1):
            j = _rand(seed + hash_key(k), i) % (i + 1)
            lst[i], lst[j] = lst[j], lst[i]
    out, rnd = [], 0
    while len(out) < count and any(strata[k] for k in keys):
        for k in keys:
            if strata[k] and len(out) < count:
                out.append(strata[k].pop())
        rnd += 1
    return out


def hash_key(k):
    h = 0
    for x in str(k).encode():
        h = (h * 131 + x) & 0xFFFFFFFF
    return h


def build_family():
    space = enumerate_space()
    core = core_set(space)
    rest = stratified_sample(space, {v["name"] for v in core}, max(0, TARGET_COUNT - len(core)), SAMPLE_SEED)
    fam = core + rest
    # The default variant (128x128x8, 8x8 threads, cp.async M-major A, VEC=1,
    # 2 stages, no split) runs every layout and alignment; it is always id 0.
    default = dict(BM=128, BN=128, BK=8, WM=32, WN=64, TM=8, TN=8, KL=1, VEC=1, STAGES=2, SPLITK=1,
                   LOADER=0, AKM=0, F2=0, fam="cpm")
    lay = lane_layout(128, 128, 8, 8, 1)
    default["WM"], default["WN"] = lay[0] * 8, lay[1] * 8
    default["name"] = name_of(default)
    fam = [default] + [v for v in fam if v["name"] != default["name"]]
    return fam, len(space)


PARAM_ORDER = ("BM", "BN", "BK", "WM", "WN", "TM", "TN", "KL", "VEC", "STAGES", "SPLITK", "LOADER", "AKM", "F2")


def params_of(v):
    return tuple(v[k] for k in PARAM_ORDER)


def row(fn, v, rid=None):
    """X-macro row: launcher index, registry id, name, template arguments."""
    return "PT_VARIANT({fn}, {rid}, \"{name}\", {args})".format(
        fn=fn, rid=fn if rid is None else rid, name=v["name"], args=", ".join(str(x) for x in params_of(v)))


def write_registry(outdir, fam, drop):
    """registry_table.inc: the family minus the variants in ``drop`` (names)."""
    rows, rid = [], 0
    for fn, v in enumerate(fam):
        if v["name"] in drop:
            continue
        rows.append(row(fn, v, rid))
        rid += 1
    text = "// generated: registered variants (%d of %d; dropped for register spills: %s)\n" % (
        rid, len(fam), ", ".join(sorted(drop)) or "none") + "\n".join(rows) + "\n"
    path = os.path.join(outdir, "registry_table.inc")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return rid


def generate(outdir):
    os.makedirs(outdir, exist_ok=True)
    fam, space_size = build_family()
    files = {}
    files["variant_table.inc"] = "// generated by gen_variants.py: %d variants of a %d-point valid space\n" % (
        len(fam), space_size) + "\n".join(row(i, v) for i, v in enumerate(fam)) + "\n"
    if not os.path.exists(os.path.join(outdir, "registry_table.inc")):
        write_registry(outdir, fam, set())
    per = (len(fam) + N_TUS - 1) // N_TUS
    for t in range(N_TUS):
        chunk = fam[t * per:(t + 1) * per]
        body = ["// generated by gen_variants.py", '#include "launch.cuh"', "",
                "#define PT_VARIANT(fn, id, name, ...) \\",
                "    int pt_launch_v##fn(const pt::GemmArgs &a, cudaStream_t s, bool dry) { \\",
                "        return pt::launch_simt<pt::Simt<__VA_ARGS__>>(a, s, dry); }", ""]
        body += [row(t * per + i, v) for i, v in enumerate(chunk)]
        files["variants_%02d.cu" % t] = "\n".join(body) + "\n"
    changed = []
    for name, text in files.items():
        path = os.path.join(outdir, name)
        if not os.path.exists(path) or open(path).read() != text:
            with open(path, "w") as f:
                f.write(text)
            changed.append(path)
    return fam, space_size, changed


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else "_gen"
    fam, n, _ = generate(out)
    print("%d variants from a valid space of %d" % (len(fam), n))
