"""Planner of the oracle (TEST INFRASTRUCTURE ONLY): ODS and PDL written out plainly.

Paper, Section 2 ("Overall Framework"):
  * ODS: an affinity graph whose nodes are the fields a section accesses and whose
    edge weights count the two fields' common occurrences; a greedy clustering
    under an architecture-dependent size limit; each cluster becomes a structure.
  * PDL: a rooted DAG over the sections with "combine" and "remap" edges; a
    shortest path through it, weighted by measured execution times, picks one
    layout per section.
Readings taken where the paper is silent (each one is listed in the design notes):
  * the weight of edge (a, b) is the number of sections of the window whose
    accessed fields (read, written, or read through the permutation) hold both;
  * greedy: edges in order (weight descending, smaller id ascending, larger id
    ascending); two clusters merge when the weight is positive and the merged
    struct (fields ascending, natural alignment) is at most `cap` bytes
    (cap <= 0: no limit); fields outside the window stay alone;
  * a layout is canonical: fields ascending within a group, groups ordered by
    their first field;
  * candidates = AoS and SoA, then the ODS layout of every window of 1..W
    consecutive sections under every cap, first occurrence kept;
  * a "combine" is two consecutive sections keeping one layout (remap cost 0);
  * the DAG is layered (input -> section 1 -> ... -> section S), so its shortest
    path is a dynamic program over the layers; among equal costs the
    lexicographically smallest sequence of layout indices wins.
"""
import itertools

from .core import group_layout, aos, soa, canon


def affinity(sections, F):
    """Edge weights {(a, b): w}, a < b: the number of record accesses, over the window's sections,
    that reach both a and b.  A section accesses its record i (the fields it reads or writes)
    and, if it gathers, the record perm[i] (the fields it reads through the permutation): two
    accesses, each adding one to every pair of its fields; a field read at i and a field read at
    perm[i] are not accessed together."""
    w = {}
    for s in sections:
        for acc in (s.read | s.write, s.read_at_perm):
            t = sorted(acc)
            for i in range(len(t)):
                for j in range(i + 1, len(t)):
                    w[(t[i], t[j])] = w.get((t[i], t[j]), 0) + 1
    return w


def ods(sections, dtypes, cap):
    """Greedy clustering of the window's affinity graph under a struct-size cap (bytes)."""
    F = len(dtypes)
    w = affinity(sections, F)
    cluster = {f: frozenset([f]) for f in range(F)}
    for (a, b), wt in sorted(w.items(), key=lambda e: (-e[1], e[0][0], e[0][1])):
        if wt <= 0 or cluster[a] is cluster[b]:
            continue
        merged = cluster[a] | cluster[b]
        _, size = group_layout(dtypes, sorted(merged))
        if cap is not None and cap > 0 and size > cap:
            continue
        for f in merged:
            cluster[f] = merged
    groups = {c for c in cluster.values()}
    return canon([sorted(c) for c in groups])


def candidates(sections, dtypes, caps, max_window=0, include_aos_soa=True, max_candidates=0):
    """Deduplicated candidate layouts in generation order."""
    F = len(dtypes)
    S = len(sections)
    out, seen = [], set()

    def add(layout):
        key = tuple(tuple(g) for g in layout)
        if key not in seen:
            seen.add(key)
            out.append(layout)

    if include_aos_soa:
        add(aos(F))
        add(soa(F))
    W = S if max_window <= 0 else min(max_window, S)
    for w in range(1, W + 1):
        for k in range(0, S - w + 1):
            for cap in caps:
                add(ods(sections[k:k + w], dtypes, cap))
    if max_candidates > 0:
        out = out[:max_candidates]
    return out


def program_cost(seq, sec_cost, remap_cost, return_to_input=False):
    """Model cost of one layout assignment: sum of section and remap costs (input layout = index L)."""
    L = len(sec_cost[0])
    total = remap_cost[L][seq[0]]
    for k, l in enumerate(seq):
        if k > 0:
            total += remap_cost[seq[k - 1]][l]
        total += sec_cost[k][l]
    if return_to_input:
        total += remap_cost[seq[-1]][L]
    return total


def pdl_exhaustive(sec_cost, remap_cost, return_to_input=False):
    """Brute force over all L^S assignments: (min cost, lexicographically smallest argmin)."""
    S, L = len(sec_cost), len(sec_cost[0])
    return min((program_cost(seq, sec_cost, remap_cost, return_to_input), list(seq))
               for seq in itertools.product(range(L), repeat=S))


def pdl_dp(sec_cost, remap_cost, return_to_input=False):
    """Shortest path through the layered DAG: (min cost, lexicographically smallest argmin).

    rest[k][l] = cheapest cost of sections k..S-1 (and the final remap) when section k
    runs in layout l; the path is then read forwards, taking the smallest index
    among the layouts that reach the minimum.
    """
    S, L = len(sec_cost), len(sec_cost[0])
    rest = [[0] * L for _ in range(S)]
    for l in range(L):
        rest[S - 1][l] = sec_cost[S - 1][l] + (remap_cost[l][L] if return_to_input else 0)
    for k in range(S - 2, -1, -1):
        for l in range(L):
            rest[k][l] = sec_cost[k][l] + min(remap_cost[l][m] + rest[k + 1][m] for m in range(L))
    seq = []
    prev = L
    for k in range(S):
        vals = [remap_cost[prev][m] + rest[k][m] for m in range(L)]
        best = min(vals)
        m = vals.index(best)
        if k == 0:
            total = best
        seq.append(m)
        prev = m
    return total, seq


# ---------------------------------------------------------------------- PDL with combine nodes
# Paper Section 2: the combine edge joins consecutive sections into one node of the DAG.  Here a
# node may be a window of m consecutive sections run in one layout (fused when m >= 2) at a
# measured cost fused_cost[(k, m)][l]; a plan is a sequence of windows (layout, length) that
# covers the sections in order.  Ties: the smaller layout, then the longer window, window by
# window from the first (the lexicographically smallest list of (layout, -length) pairs).

def fused_program_cost(windows, sec_cost, remap_cost, fused_cost, return_to_input=False):
    """Model cost of one plan given as [(layout, length), ...] (input layout = index L)."""
    L = len(sec_cost[0])
    prev, k, total = L, 0, 0
    for l, m in windows:
        total += remap_cost[prev][l] + (sec_cost[k][l] if m == 1 else fused_cost[(k, m)][l])
        prev, k = l, k + m
    if return_to_input:
        total += remap_cost[prev][L]
    return total


def _compositions(S, W):
    """Every way to cut S sections into consecutive windows of 1..W sections."""
    if S == 0:
        yield []
        return
    for m in range(1, min(W, S) + 1):
        for rest in _compositions(S - m, W):
            yield [m] + rest


def _as_plan(windows, S):
    seq, win = [], []
    for l, m in windows:
        seq += [l] * m
        win += [m] + [0] * (m - 1)
    return seq, win


def pdl_exhaustive_fused(sec_cost, remap_cost, fused_cost, max_window, return_to_input=False):
    """Brute force over every cut into windows and every layout per window:
    (min cost, layout per section, window length at each window's first section and 0 inside)."""
    S, L = len(sec_cost), len(sec_cost[0])
    best = None
    for cut in _compositions(S, max(1, max_window)):
        for lays in itertools.product(range(L), repeat=len(cut)):
            windows = list(zip(lays, cut))
            key = (fused_program_cost(windows, sec_cost, remap_cost, fused_cost, return_to_input),
                   [(l, -m) for l, m in windows])
            if best is None or key < best[0]:
                best = (key, windows)
    seq, win = _as_plan(best[1], S)
    return best[0][0], seq, win


def pdl_dp_fused(sec_cost, remap_cost, fused_cost, max_window, return_to_input=False):
    """Shortest path with combine nodes: (min cost, layout per section, window lengths).

    rest[k][p] = cheapest cost of sections k..S-1 (and the final remap) when the data is in
    layout p before section k (p = L: the input layout); the path is read forwards, taking
    the smallest layout, then the longest window, among the choices that reach the minimum.
    """
    S, L = len(sec_cost), len(sec_cost[0])
    W = max(1, max_window)

    def cost(k, m, l):
        return sec_cost[k][l] if m == 1 else fused_cost[(k, m)][l]

    rest = [[0] * (L + 1) for _ in range(S + 1)]
    for p in range(L + 1):
        rest[S][p] = remap_cost[p][L] if return_to_input else 0
    choices = lambda k, p: [(remap_cost[p][l] + cost(k, m, l) + rest[k + m][l], l, -m)
                            for l in range(L) for m in range(1, min(W, S - k) + 1)]
    for k in range(S - 1, -1, -1):
        for p in range(L + 1):
            rest[k][p] = min(c[0] for c in choices(k, p))
    windows, p, k = [], L, 0
    while k < S:
        c, l, negm = min(choices(k, p))
        windows.append((l, -negm))
        p, k = l, k - negm
    seq, win = _as_plan(windows, S)
    return rest[0][L], seq, win


# ---------------------------------------------------------------------- PDL over a structured CFG
# Paper Section 2: PDL builds a rooted DAG from the program's structured control-flow graph
# (SCFG) and takes a shortest path through it.  The paper gives no cost rule for branches and
# loops; the reading here: a program is a tree of regions
#   ("sec", k)                       section k of the cost table,
#   ("seq", [regions])               regions one after another (an empty one changes nothing),
#   ("branch", [regions], [w])       one of the regions runs, region b with probability w[b]
#                                    (the w sum to 1); the branches meet again at a merge point,
#   ("loop", region, T)              the region runs T >= 1 times (a loop tested at its end),
# (regions are lists or tuples, each a distinct object: plans are keyed by the region's identity)
# and a plan gives a layout to every section, to every merge point and to every loop header
# (the layout the data is in whenever an iteration starts); layout index L is the input layout,
# which merge points and headers may also keep.  The cost is the expected time: every section
# and every remap on the way weighted by how often it runs; a branch's path pays the remap from
# its last layout to the merge point's; an iteration starts with the remap into the header's
# layout (from the entry layout the first time, from the body's last layout after that).

INF = float("inf")


def scfg_nodes(tree):
    """The regions of a tree in preorder: [(kind, payload)], children before their next sibling."""
    out = []

    def walk(t):
        out.append(t)
        if t[0] == "seq":
            for c in t[1]:
                walk(c)
        elif t[0] == "branch":
            for c in t[1]:
                walk(c)
        elif t[0] == "loop":
            walk(t[1])
    walk(tree)
    return out


def scfg_expected_cost(tree, layout, sec_cost, remap_cost, return_to_input=False):
    """Expected cost of a plan: `layout` maps id(region) -> layout of that section / merge point /
    loop header.  Evaluated by following the regions with their execution weights."""
    L = len(sec_cost[0])

    def run(t, cur):                  # (expected cost, layout afterwards)
        kind = t[0]
        if kind == "sec":
            l = layout[id(t)]
            return remap_cost[cur][l] + sec_cost[t[1]][l], l
        if kind == "seq":
            total = 0
            for c in t[1]:
                cost, cur = run(c, cur)
                total += cost
            return total, cur
        if kind == "branch":
            m = layout[id(t)]
            total = 0
            for c, w in zip(t[1], t[2]):
                cost, out = run(c, cur)
                total += w * (cost + remap_cost[out][m])
            return total, m
        f = layout[id(t)]             # loop header
        body, T = t[1], t[2]
        cost, out = run(body, f)
        return remap_cost[cur][f] + T * cost + (T - 1) * remap_cost[out][f], out

    total, out = run(tree, L)
    if return_to_input:
        total += remap_cost[out][L]
    return total


def pdl_scfg_exhaustive(tree, sec_cost, remap_cost, return_to_input=False):
    """Brute force over every layout of every section (0..L-1), merge point and loop header
    (0..L): the least expected cost."""
    L = len(sec_cost[0])
    nodes = [t for t in scfg_nodes(tree) if t[0] in ("sec", "branch", "loop")]
    choices = [range(L) if t[0] == "sec" else range(L + 1) for t in nodes]
    best = None
    for assign in itertools.product(*choices):
        cost = scfg_expected_cost(tree, {id(t): l for t, l in zip(nodes, assign)}, sec_cost, remap_cost,
                                  return_to_input)
        if best is None or cost < best:
            best = cost
    return best


def _minplus(A, B):
    n, m, k = len(A), len(B[0]), len(B)
    return [[min(A[i][q] + B[q][j] for q in range(k)) for j in range(m)] for i in range(n)]


def pdl_scfg_dp(tree, sec_cost, remap_cost, return_to_input=False):
    """Shortest expected path over the SCFG by dynamic programming on the region tree: every
    region gets a matrix C[p][q] = least expected cost of running it entered in layout p and
    left in layout q (0..L, L = input layout).  A section: the remap into its layout plus its
    cost; a sequence: the min-plus product of its regions' matrices; a branch: for a merge
    layout q, the sum over branches of w_b * min over the branch's last layout (its matrix plus
    the remap to q); a loop with header f: remap into f, T times the body from f, T - 1 remaps
    from the body's last layout back to f, the least over f.  Returns (least expected cost,
    {id(region): layout}) for one best plan."""
    L = len(sec_cost[0])
    N = L + 1
    rem = remap_cost
    memo = {}

    def mat(t):
        key = id(t)
        if key in memo:
            return memo[key]
        kind = t[0]
        if kind == "sec":
            k = t[1]
            C = [[rem[p][q] + sec_cost[k][q] if q < L else INF for q in range(N)] for p in range(N)]
        elif kind == "seq":
            C = [[0 if p == q else INF for q in range(N)] for p in range(N)]
            for c in t[1]:
                C = _minplus(C, mat(c))
        elif kind == "branch":
            C = [[0.0] * N for _ in range(N)]
            for c, w in zip(t[1], t[2]):
                B = mat(c)
                for p in range(N):
                    for q in range(N):
                        C[p][q] += w * min(B[p][r] + rem[r][q] for r in range(N))
        else:
            B, T = mat(t[1]), t[2]
            C = [[min(rem[p][f] + T * B[f][e] + (T - 1) * rem[e][f] for f in range(N)) for e in range(N)]
                 for p in range(N)]
        memo[key] = C
        return C

    plan = {}

    def pick(t, p, q):   # record the choices of one best path through t entered in p, left in q
        kind = t[0]
        if kind == "sec":
            plan[id(t)] = q
        elif kind == "seq":
            cs = t[1]
            # prefix products, then walk back choosing each intermediate layout
            pref = [[[0 if a == b else INF for b in range(N)] for a in range(N)]]
            for c in cs:
                pref.append(_minplus(pref[-1], mat(c)))
            cur = q
            for i in range(len(cs), 0, -1):
                M = mat(cs[i - 1])
                prev = min(range(N), key=lambda r: pref[i - 1][p][r] + M[r][cur])
                pick(cs[i - 1], prev, cur)
                cur = prev
        elif kind == "branch":
            plan[id(t)] = q
            for c in t[1]:
                B = mat(c)
                r = min(range(N), key=lambda r: B[p][r] + rem[r][q])
                pick(c, p, r)
        else:
            B, T = mat(t[1]), t[2]
            f = min(range(N), key=lambda f: rem[p][f] + T * B[f][q] + (T - 1) * rem[q][f])
            plan[id(t)] = f
            pick(t[1], f, q)

    C = mat(tree)
    ends = [C[L][q] + (rem[q][L] if return_to_input else 0) for q in range(N)]
    q = min(range(N), key=lambda q: ends[q])
    pick(tree, L, q)
    return ends[q], plan


# ---------------------------------------------------------------------- PDL with a device dimension
# Paper Section 2 and Table 4: PDL maps every section to a device as well as a layout (Medical:
# CPU-ODS(1-3) remap GPU-ODS(4-7)).  The reading here: D devices, each with its own cost table
# (section times and remap times between layouts on that device, input layout = index L) and a
# transfer time xfer[a][b][l] for moving data in layout l from device a to device b (l = L: the
# input layout).  A plan gives each section a (layout, device); between consecutive sections on
# one device the edge is that device's remap; across devices it is the cheaper of remapping on
# the source then moving the result, or moving the data then remapping on the destination.  The
# input starts in layout L on input_device; return_to_input adds the way back to it.

def device_edge(rem, xfer, a, la, b, lb):
    """Cost of going from layout la on device a to layout lb on device b."""
    if a == b:
        return rem[a][la][lb]
    return min(rem[a][la][lb] + xfer[a][b][lb], xfer[a][b][la] + rem[b][la][lb])


def device_program_cost(plan, sec, rem, xfer, input_device, return_to_input=False):
    """Model cost of a plan [(layout, device), ...]; sec[d][k][l], rem[d][a][b], xfer[a][b][l]."""
    L = len(sec[0][0])
    cur = (L, input_device)
    total = 0
    for k, (l, d) in enumerate(plan):
        total += device_edge(rem, xfer, cur[1], cur[0], d, l) + sec[d][k][l]
        cur = (l, d)
    if return_to_input:
        total += device_edge(rem, xfer, cur[1], cur[0], input_device, L)
    return total


def pdl_devices_exhaustive(sec, rem, xfer, input_device, return_to_input=False):
    """Brute force over every (layout, device) per section: (least cost, smallest such plan)."""
    D, S, L = len(sec), len(sec[0]), len(sec[0][0])
    states = [(l, d) for d in range(D) for l in range(L)]
    return min((device_program_cost(list(p), sec, rem, xfer, input_device, return_to_input), list(p))
               for p in itertools.product(states, repeat=S))


def pdl_devices_dp(sec, rem, xfer, input_device, return_to_input=False):
    """The layered-DAG shortest path over (layout, device) states (state index d*L + l), ties to
    the smaller state index: (least cost, [(layout, device)] per section)."""
    D, S, L = len(sec), len(sec[0]), len(sec[0][0])
    states = [(l, d) for d in range(D) for l in range(L)]
    n = len(states)
    edge = lambda x, y: device_edge(rem, xfer, x[1], x[0], y[1], y[0])
    start = (L, input_device)
    rest = [[0] * n for _ in range(S)]
    for i, (l, d) in enumerate(states):
        rest[S - 1][i] = sec[d][S - 1][l] + (edge((l, d), start) if return_to_input else 0)
    for k in range(S - 2, -1, -1):
        for i, (l, d) in enumerate(states):
            rest[k][i] = sec[d][k][l] + min(edge((l, d), states[j]) + rest[k + 1][j] for j in range(n))
    plan, prev, total = [], start, None
    for k in range(S):
        vals = [edge(prev, states[j]) + rest[k][j] for j in range(n)]
        j = vals.index(min(vals))
        if k == 0:
            total = vals[j]
        plan.append(states[j])
        prev = states[j]
    return total, plan
