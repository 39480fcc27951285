"""Models, in plain Python, of the two parallel resolutions of the type-2 deflation scan
(Section 3.2), each checked against the sequential scan it replaces, on random poles with
runs of equal values (chains of rotations, which the speculation does not cover), on
isolated equal pairs (the pattern of symmetric halves) and on poles whose test against a
rotated survivor passes where the test on the original values fails.  Each of three
plausible mistakes (the bit-mask shortcut without its bit-1 condition, a chain's state
reset after a rotation, the band scan trusting the speculation after a rotation) fails
one of the two tests.

The scan walks the survivors of the type-1 test in order with a candidate p: the pair
(p, j) rotates when |(D_j - D_p) c s| <= tol (c = z_j / tau, s = -z_p / tau,
tau = hypot); the rotated survivor j (with its new value and weight) becomes the
candidate, p is deflated; otherwise p is kept and j becomes the candidate.

* The merge's resolution (k_prepare): every pair is tested in parallel on the original
  values (bit 0) and, after a bit-0 rotation, the next pair against the rotated survivor
  (bit 1); a warp then decides 32 poles at a time with a three-state machine (N: the
  candidate is an original pole, S: it came from a bit-0 rotation, X: from any other
  rotation, tested in FP64), or, when no bit-0 rotation follows a rotation and no pole
  after one has bit 1, takes the bit-0 word as the decisions; each pole's record (index,
  candidate, candidate support, values) then follows from the decision word.
* The band merge's resolution (k_bd_deflate): the same speculative test, one thread
  jumping from one speculative rotation to the next and testing a pair itself only right
  after a rotation; kept and deflated lists compacted afterwards.

Verification only: the models fix the decision rules; the GPU tests check the kernels'
results and deflation counts against the oracle."""
import math
import random


def t2test(D, z, pD, pz, tol):
    return abs((D - pD) * z * pz) <= tol * (z * z + pz * pz)


def t2rot(D, z, pD, pz):
    t2 = z * z + pz * pz
    r = 1.0 / math.sqrt(t2)
    cc, ss, tau = z * r, -pz * r, t2 * r
    c2, s2 = cc * cc, ss * ss
    return cc, ss, tau, pD * c2 + D * s2, pD * s2 + D * c2  # c, s, new weight, deflated, new pole


def speculate(D, z, tol):
    n = len(D)
    f, spec = [0] * n, [None] * n
    for q in range(1, n):
        if t2test(D[q], z[q], D[q - 1], z[q - 1], tol):
            f[q] |= 1
            spec[q] = t2rot(D[q], z[q], D[q - 1], z[q - 1])
    for q in range(2, n):
        if f[q - 1] & 1 and t2test(D[q], z[q], spec[q - 1][4], spec[q - 1][2], tol):
            f[q] |= 2
    return f, spec


def merge_sequential(D, z, c, sp, f, spec, tol):
    """The one-thread resolution: per pole a record (kind, code, index, chain index,
    candidate, support, values) and the final candidate."""
    rec, K, nr, nch = {}, 0, 0, 0
    pj, pD, pz, ps, prev_rot, prev_simple = -1, 0.0, 0.0, 0, False, False
    for q in range(len(D)):
        if q == 0:
            pj, pD, pz, ps, prev_rot = c[0], D[0], z[0], sp[0], False
            continue
        if not prev_rot:
            rot = bool(f[q] & 1)
            if rot:
                cc, ss, tau, dp, di = spec[q]
            prev_simple = rot
        else:
            rot = bool(f[q] & 2) if prev_simple else t2test(D[q], z[q], pD, pz, tol)
            if rot:
                cc, ss, tau, dp, di = t2rot(D[q], z[q], pD, pz)
            prev_simple = False
        if rot:
            rec[q] = ("rot", 1 if prev_rot else 3, nr, None if prev_rot else nch, pj, ps | (sp[q] << 8), (cc, ss, dp))
            nr += 1
            nch += 0 if prev_rot else 1
            pj, pD, pz, ps, prev_rot = c[q], di, tau, ps | sp[q], True
        else:
            rec[q] = ("keep", 0, K, None, pj, ps, (pD, pz))
            K += 1
            pj, pD, pz, ps, prev_rot = c[q], D[q], z[q], sp[q], False
    return rec, K, nr, nch, ((pj, pD, pz, ps) if pj >= 0 else None)


def merge_warp(D, z, c, sp, f, spec, tol):
    """The warp-level resolution, 32 poles at a time."""
    n = len(D)
    sc = {q: list(spec[q]) if spec[q] else None for q in range(n)}  # staged values; recomputed ones overwrite
    rec, K, nr, nch = {}, 0, 0, 0
    st, cpj, cpD, cpz, cps, cprot = "N", -1, 0.0, 0.0, 0, False
    for q0 in range(0, n, 32):
        kn = min(32, n - q0)
        b0 = sum(1 << i for i in range(kn) if q0 + i > 0 and f[q0 + i] & 1)
        b1 = sum(1 << i for i in range(kn) if q0 + i > 0 and f[q0 + i] & 2)
        kmask = (1 << kn) - 1
        sS = ((b0 << 1) & 0xFFFFFFFF) | (1 if st == "S" else 0)
        rotw, s = 0, st
        if st != "X" and (b0 & sS) == 0 and (b1 & sS & kmask) == 0:
            rotw, s = b0, ("S" if (b0 >> (kn - 1)) & 1 else "N")
        else:
            k = 0
            while k < kn:
                q = q0 + k
                if q == 0:
                    s, k = "N", k + 1
                    continue
                if s == "N":
                    m = b0 >> k
                    if m == 0:
                        break
                    k += (m & -m).bit_length() - 1
                    rotw |= 1 << k
                    s, k = "S", k + 1
                    continue
                if s == "S" and not (b1 >> k) & 1:
                    s, k = "N", k + 1
                    continue
                pDv, pzv = (sc[q - 1][4], sc[q - 1][2]) if k > 0 else (cpD, cpz)
                if s == "S" or t2test(D[q], z[q], pDv, pzv, tol):
                    sc[q] = list(t2rot(D[q], z[q], pDv, pzv))
                    rotw |= 1 << k
                    s = "X"
                else:
                    s = "N"
                k += 1
        prevw = ((rotw << 1) | (1 if cprot else 0)) & kmask
        starts = rotw & ~prevw
        keepw = ~rotw & kmask & (~1 if q0 == 0 else ~0)
        top = sum(1 << i for i in range(kn) if sp[q0 + i] == 1)
        bot = sum(1 << i for i in range(kn) if sp[q0 + i] == 2)

        def run_sup(m):  # OR of the supports over the run of rotations ending at index m
            upto = (2 << m) - 1
            zeros = ~rotw & upto
            extra, rng = cps, upto
            if zeros:
                rng, extra = upto & ~((1 << (zeros.bit_length() - 1)) - 1), 0
            return extra | (1 if top & rng else 0) | (2 if bot & rng else 0)

        for lane in range(kn):
            q = q0 + lane
            if q == 0:
                continue
            lt = (1 << lane) - 1
            rot, prot = (rotw >> lane) & 1, (prevw >> lane) & 1
            ps = run_sup(lane - 1) if lane > 0 else cps
            pj = c[q - 1] if lane > 0 else cpj
            if rot:
                cc, ss, _, dp, _ = sc[q]
                rec[q] = ("rot", 1 if prot else 3, nr + bin(rotw & lt).count("1"),
                          None if prot else nch + bin(starts & lt).count("1"), pj, ps | (sp[q] << 8), (cc, ss, dp))
            else:
                if lane == 0:
                    vals = (cpD, cpz)
                else:
                    vals = (sc[q - 1][4], sc[q - 1][2]) if prot else (D[q - 1], z[q - 1])
                rec[q] = ("keep", 0, K + bin(keepw & lt).count("1"), None, pj, ps, vals)
        last = kn - 1
        lr = (rotw >> last) & 1
        cps, cpj, cprot, st = run_sup(last), c[q0 + last], bool(lr), s
        cpD, cpz = (sc[q0 + last][4], sc[q0 + last][2]) if lr else (D[q0 + last], z[q0 + last])
        K += bin(keepw).count("1")
        nr += bin(rotw).count("1")
        nch += bin(starts).count("1")
    return rec, K, nr, nch, ((cpj, cpD, cpz, cps) if n > 0 else None)


def band_sequential(D, z, tol):
    kept, defl, rot, pj = [], [], [], -1
    D, z = list(D), list(z)
    for j in range(len(D)):
        if pj < 0:
            pj = j
            continue
        s, c = z[pj], z[j]
        tau = math.hypot(c, s)
        c, s = c / tau, -s / tau
        if abs((D[j] - D[pj]) * c * s) <= tol:
            z[j], z[pj] = tau, 0.0
            rot.append((pj, j, c, s))
            dp, dn = D[pj], D[j]
            D[pj], D[j] = dp * c * c + dn * s * s, dp * s * s + dn * c * c
            defl.append(pj)
        else:
            kept.append(pj)
        pj = j
    if pj >= 0:
        kept.append(pj)
    return kept, defl, rot, D, z


def band_jumping(D, z, tol):
    D, z = list(D), list(z)
    M = len(D)
    bits, spec = [False] * (M + 1), {}
    for q in range(1, M):
        zp, zj, dp, dj = z[q - 1], z[q], D[q - 1], D[q]
        w = math.hypot(zj, zp)
        c, s = zj / w, -zp / w
        bits[q] = abs((dj - dp) * c * s) <= tol
        spec[q] = (c, s, w, dp * c * c + dj * s * s, dp * s * s + dj * c * c)
    dbit, rot, mod, zc, dc, q = [False] * M, [], False, 0.0, 0.0, 1
    slot = [-1] * M
    while q < M:
        if not mod:
            nxt = [k for k in range(q, M) if bits[k]]
            if not nxt:
                break
            q = nxt[0]
            r, (c, s, w, dp, dn) = True, spec[q]
        else:
            w = math.hypot(z[q], zc)
            c, s = z[q] / w, -zc / w
            r = abs((D[q] - dc) * c * s) <= tol
            dp, dn = dc * c * c + D[q] * s * s, dc * s * s + D[q] * c * c
        if r:
            z[q], z[q - 1], D[q - 1], D[q] = w, 0.0, dp, dn
            rot.append((q - 1, q, c, s))
            slot[q], dbit[q - 1], mod, zc, dc = q - 1, True, True, w, dn
        else:
            mod = False
        q += 1
    kept = [q for q in range(M) if not dbit[q]]
    defl = [e for e in slot if e >= 0]
    return kept, defl, rot, D, z


def poles(rnd, n, pairs, sticky=False):
    """Sorted poles and weights: runs of equal or nearly equal values (pairs=False), isolated
    equal pairs (pairs=True), or (sticky=True) pairs of equal poles with weights (1, 1e-6)
    followed by a pole 1e-11 above with weight 1e-6, whose test fails on the original
    values and passes against the rotated survivor (bit 1 without bit 0)."""
    if sticky:
        D, z, x = [], [], 0.0
        while len(D) < n:
            x += rnd.random() + 0.1
            if rnd.random() < 0.7:
                D += [x, x, x + 1e-11]
                z += [1.0, 1e-6, 1e-6]
            else:
                D.append(x)
                z.append(rnd.uniform(0.1, 1.0))
        return D[:n], z[:n]
    D, x = [], 0.0
    while len(D) < n:
        if pairs:
            x += rnd.random() + 0.1
            D += [x] * (1 + (rnd.random() < 0.8) + (rnd.random() < 0.03))
        else:
            r = rnd.random()
            x += 0.0 if (r < 0.35 and D) else (1e-17 if r < 0.5 else rnd.random())
            D.append(x)
    D = D[:n]
    z = [rnd.uniform(0.1, 1.0) if pairs else rnd.uniform(-1, 1) * (1e-9 if rnd.random() < 0.1 else 1.0)
         for _ in range(n)]
    return D, z


def test_warp_resolution_equals_the_sequential_scan():
    rotations = chains = 0
    for seed in range(1200):
        rnd = random.Random(seed)
        n = rnd.randint(0, 200)
        D, z = poles(rnd, n, pairs=seed % 3 == 1, sticky=seed % 3 == 2)
        c = list(range(n))
        rnd.shuffle(c)
        sp = [1 if ci < n // 2 else 2 for ci in c]
        f, spec = speculate(D, z, 1e-12)
        a = merge_sequential(D, z, c, sp, f, spec, 1e-12)
        assert merge_warp(D, z, c, sp, f, spec, 1e-12) == a, seed
        rotations += a[2]
        chains += sum(1 for r in a[0].values() if r[0] == "rot" and r[1] == 1)
    assert rotations > 50000 and chains > 1000  # both paths of the state machine were taken


def test_band_resolution_equals_the_sequential_scan():
    rotations = 0
    for seed in range(600):
        rnd = random.Random(10 ** 6 + seed)
        n = rnd.randint(1, 200)
        D, z = poles(rnd, n, pairs=seed % 3 == 1, sticky=seed % 3 == 2)
        a = band_sequential(D, z, 1e-12)
        assert band_jumping(D, z, 1e-12) == a, seed
        rotations += len(a[2])
    assert rotations > 10000
