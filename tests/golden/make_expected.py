"""Writes stored expected results for workloads too slow for the oracle to
run inside the test suite.  Calls only the CPU oracle and the seeded input
generators; nothing here touches the CUDA library.

    python tests/golden/make_expected.py snn16k     # 16,384-node SNN, Omega 2^10, Delta 2^12
    python tests/golden/make_expected.py batch64    # 39 members of the 64-instance batch
    python tests/golden/make_expected.py batch64 4,52,30 --jobs 6
        # more members, one oracle run per worker process, merged into the file

Output: tests/golden/expected_<name>.txt with the Eq. (1) cost, the number of
parts, the number of levels, the per-level node counts, and a SHA-256 of
the part ids (int32 little-endian) and of the per-part (weight, inbound)
pairs.
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

WORKLOADS = {
    "snn16k": (lambda: synth.snn_16k(0), 1024, 4096),
    "snn4k": (lambda: synth.random_snn(4096, 64, 0), 256, 1024),
}


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# members of synth.batch_instances(64, 0) the oracle finishes in minutes, all
# at Omega 2^10, Delta 2^12: every conv-style member (odd index, 2k-59k
# nodes, up to 11.9 M pins) and seven random ones (3k-5k nodes)
BATCH_MEMBERS = tuple(range(1, 64, 2)) + (6, 0, 42, 32, 40, 24, 48)


def batch64():
    inst = synth.batch_instances(64, 0)
    path = os.path.join(ROOT, "tests", "golden", "expected_batch64.txt")
    lines = ["# oracle results for members of the 64-instance batch (seed 0), omega=1024, delta=4096",
             "# written by tests/golden/make_expected.py batch64",
             "# member: cost num_parts num_levels sha_part_ids sha_part_stats"]
    for i in BATCH_MEMBERS:
        g = inst[i]
        t = time.time()
        with oracle.Run.from_graph(g) as r:
            res = r.partition(1024, 4096)
            nlev = r.num_levels
        stats = np.stack([res.part_weight.astype(np.int64), res.part_inbound.astype(np.int64)], axis=1)
        lines.append(f"{i}: {res.cost} {res.num_parts} {nlev} {digest(res.part_ids.astype('<i4'))} "
                     f"{digest(stats.astype('<i8'))}  # {g.name}, {time.time() - t:.0f} s")
        print(lines[-1], flush=True)
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(path)


def _member_line(i):
    """One member's result line (runs in a worker process)."""
    g = synth.batch_instances(64, 0)[i]
    t = time.time()
    with oracle.Run.from_graph(g) as r:
        res = r.partition(1024, 4096)
        nlev = r.num_levels
    stats = np.stack([res.part_weight.astype(np.int64), res.part_inbound.astype(np.int64)], axis=1)
    return i, (f"{i}: {res.cost} {res.num_parts} {nlev} {digest(res.part_ids.astype('<i4'))} "
               f"{digest(stats.astype('<i8'))}  # {g.name}, {time.time() - t:.0f} s")


def batch64_more(members, jobs):
    """Adds the listed members to expected_batch64.txt, keeping the lines
    already there; each finished member is written at once."""
    import concurrent.futures as cf
    import multiprocessing as mp
    path = os.path.join(ROOT, "tests", "golden", "expected_batch64.txt")
    with cf.ProcessPoolExecutor(max_workers=jobs, mp_context=mp.get_context("spawn")) as ex:
        for fut in cf.as_completed([ex.submit(_member_line, i) for i in members]):
            i, line = fut.result()
            with open(path) as f:
                lines = [l.rstrip("\n") for l in f]
            head = [l for l in lines if l.startswith("#")]
            body = {int(l.split(":", 1)[0]): l for l in lines if l and not l.startswith("#")}
            body[i] = line
            with open(path, "w") as f:
                f.write("\n".join(head + [body[k] for k in sorted(body)]) + "\n")
            print(line, flush=True)


def main(name: str):
    if name == "batch64":
        if len(sys.argv) > 2:
            jobs = int(sys.argv[sys.argv.index("--jobs") + 1]) if "--jobs" in sys.argv else 1
            return batch64_more([int(x) for x in sys.argv[2].split(",")], jobs)
        return batch64()
    make, omega, delta = WORKLOADS[name]
    g = make()
    t = time.time()
    with oracle.Run.from_graph(g) as r:
        res = r.partition(omega, delta)
        levels = [r.level_V(l) for l in range(r.num_levels)]
    secs = time.time() - t
    stats = np.stack([res.part_weight.astype(np.int64), res.part_inbound.astype(np.int64)], axis=1)
    path = os.path.join(ROOT, "tests", "golden", f"expected_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# oracle result for {g.name}, omega={omega}, delta={delta}\n")
        f.write(f"# written by tests/golden/make_expected.py ({secs:.0f} s of oracle time)\n")
        f.write(f"omega: {omega}\ndelta: {delta}\ncost: {res.cost}\nnum_parts: {res.num_parts}\n")
        f.write(f"num_levels: {len(levels)}\n")
        f.write("level_V: " + " ".join(str(v) for v in levels) + "\n")
        f.write(f"sha_part_ids: {digest(res.part_ids.astype('<i4'))}\n")
        f.write(f"sha_part_stats: {digest(stats.astype('<i8'))}\n")
    print(path, res.cost, res.num_parts, len(levels), f"{secs:.0f}s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "snn16k")
