"""The runner's tile-map check on the CPU (csrc/runner_bounds.h), compiled
here with the host compiler.

The persistent multi-lattice kernel maps a global tile number to (phase,
lattice, tile) through three host-built tables and does no bounds checks of
its own; lat_runner_run checks the tables first and returns LAT_ESTATE
instead of launching.  Maps built the way the runner builds them must pass,
and each kind of inconsistency the kernel could index out of bounds with
must be rejected.
"""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_18624_gb300", "csrc")
THREADS = 256


@pytest.fixture(scope="module")
def check(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("maps") / "runner_maps_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC,
                           os.path.join(ROOT, "tests", "cpp", "runner_maps_check.cpp"), "-o", exe])

    def run(maps):
        lines = []
        for m in maps:
            n, K = len(m["desc"]), len(m["hact"])
            lines.append("%d %d %d" % (n, K, m.get("threads", THREADS)))
            lines += ["%d %d %d" % d for d in m["desc"]]
            lines.append(" ".join(map(str, m["htp"])))
            lines.append(" ".join(map(str, m["hpb"])))
            lines.append(" ".join(map(str, m["hact"])))
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split()
        assert len(out) == len(maps)
        return [o == "1" for o in out]
    return run


def build(items, tiles, nsweeps):
    """The maps as the runner builds them: lattices by descending sweep
    count, ntiles = ceil(items / tile), a lattice active in phase k while
    k < 2 * nsweeps."""
    order = sorted(range(len(items)), key=lambda i: -nsweeps[i])
    desc = [(items[i], tiles[i], -(-items[i] // tiles[i])) for i in order]
    htp = [0]
    for d in desc:
        htp.append(htp[-1] + d[2])
    K = 2 * max(nsweeps)
    hact, hpb = [], [0]
    for k in range(K):
        act = sum(1 for i in order if 2 * nsweeps[i] > k)
        hact.append(act)
        hpb.append(hpb[-1] + htp[act])
    return {"desc": desc, "htp": htp, "hpb": hpb, "hact": hact}


def random_maps(rng):
    n = int(rng.integers(1, 9))
    items = [int(rng.integers(1, 1 << 22)) for _ in range(n)]
    tiles = [THREADS * int(rng.integers(1, 65)) for _ in range(n)]
    nsweeps = [int(rng.integers(1, 6)) for _ in range(n)]
    return build(items, tiles, nsweeps)


def _consistent(c):
    """Recompute the prefix tables from desc and hact (where hact allows), so
    that an edit of desc or hact breaks only the condition it targets."""
    n = len(c["desc"])
    c["htp"] = [0]
    for d in c["desc"]:
        c["htp"].append(c["htp"][-1] + d[2])
    c["hpb"] = [0]
    for a in c["hact"]:
        c["hpb"].append(c["hpb"][-1] + (c["htp"][a] if 0 <= a <= n else 0))


def mutations(m):
    """Copies of m, each with one inconsistency."""
    out = []

    def edit(fn, recompute=True):
        c = {k: [tuple(x) for x in v] if k == "desc" else list(v) for k, v in m.items()}
        fn(c)
        if recompute:
            _consistent(c)
        out.append(c)

    n, K = len(m["desc"]), len(m["hact"])
    s = n - 1
    items, tile, nt = m["desc"][s]
    edit(lambda c: c["desc"].__setitem__(s, (items, 0, nt)))                    # empty tiles
    edit(lambda c: c["desc"].__setitem__(s, (items, tile + THREADS // 2, nt)))  # tile not a block multiple
    edit(lambda c: c["desc"].__setitem__(s, (items, tile, 0)))                  # no tiles
    if nt > 1:
        edit(lambda c: c["desc"].__setitem__(s, (items, tile, nt - 1)))         # items left uncovered
    edit(lambda c: c["desc"].__setitem__(s, (items, tile, nt + 1)))             # a tile past the items
    edit(lambda c: c["htp"].__setitem__(0, 1), recompute=False)                 # prefix not from 0
    edit(lambda c: c["htp"].__setitem__(n, c["htp"][n] + 1), recompute=False)   # prefix off by one

    def prefix_only(c):  # the prefix disagrees with the tile counts, the phase bases agree with the prefix
        c["htp"][n] += 1
        c["hpb"] = [0]
        for a in c["hact"]:
            c["hpb"].append(c["hpb"][-1] + c["htp"][a])
    edit(prefix_only, recompute=False)
    edit(lambda c: c["hpb"].__setitem__(0, 1), recompute=False)                 # phase bases not from 0
    edit(lambda c: c["hpb"].__setitem__(K, c["hpb"][K] - 1), recompute=False)   # phase base off by one
    edit(lambda c: c["hact"].__setitem__(K - 1, 0))                             # a phase with no lattice
    edit(lambda c: c["hact"].__setitem__(0, n + 1))                             # more active than lattices
    if n > 1 and K > 1:
        def grow(c):                                                             # active count grows
            c["hact"][0], c["hact"][1] = 1, 2
        edit(grow)
    return out


def test_maps_built_like_the_runner_pass(check):
    rng = np.random.default_rng(5)
    maps = [random_maps(rng) for _ in range(300)]
    maps.append(build([256], [256], [1]))                       # one tile, one sweep
    maps.append(build([1 << 22, 300], [4096, 512], [3, 3]))     # equal sweep counts
    maps.append(build([17] * 8, [256] * 8, [1, 2, 3, 4, 5, 6, 7, 8]))
    assert all(check(maps))


def test_each_inconsistency_is_rejected(check):
    rng = np.random.default_rng(6)
    cases = []
    for _ in range(100):
        cases += mutations(random_maps(rng))
    cases += mutations(build([1 << 20, 1 << 16, 4096], [4096, 512, 256], [4, 2, 2]))
    got = check(cases)
    bad = [c for c, g in zip(cases, got) if g]
    assert not bad, bad[:2]


@pytest.mark.parametrize("old,new", [
    ("d.tile_items % threads != 0 || ", ""),
    (" || (uint64_t)(d.ntiles - 1) * d.tile_items >= d.items", ""),
    ("(uint64_t)d.ntiles * d.tile_items < d.items || ", ""),
    (" || (k > 0 && hact[k] > hact[k - 1])", ""),
    ("if ((uint64_t)htp[s + 1] != (uint64_t)htp[s] + d.ntiles) return false;", ""),
])
def test_a_check_taken_out_lets_an_inconsistency_through(tmp_path, old, new):
    """Planted mistakes in a copy of the check: each condition is the only
    one that rejects some inconsistent map."""
    with open(os.path.join(CSRC, "runner_bounds.h")) as f:
        src = f.read()
    assert src.count(old) == 1, old
    inc = tmp_path / "inc"
    inc.mkdir()
    (inc / "runner_bounds.h").write_text(src.replace(old, new))
    exe = str(tmp_path / "runner_maps_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", str(inc),
                           os.path.join(ROOT, "tests", "cpp", "runner_maps_check.cpp"), "-o", exe])
    rng = np.random.default_rng(6)
    cases = []
    for _ in range(100):
        cases += mutations(random_maps(rng))
    lines = []
    for m in cases:
        lines.append("%d %d %d" % (len(m["desc"]), len(m["hact"]), THREADS))
        lines += ["%d %d %d" % d for d in m["desc"]]
        lines += [" ".join(map(str, m[k])) for k in ("htp", "hpb", "hact")]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split()
    assert "1" in out, "no inconsistent map got through without: %s" % old
