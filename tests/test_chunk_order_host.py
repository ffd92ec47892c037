"""Host-side check of the bit-packed classifiers' chunk order (ChunkWalk in
rsr_internal.cuh, a __host__ __device__ struct), compiled for the host with
nvcc: every chunk of both sets is visited exactly once, in increasing index
within each set; with an overlapping pair every lower chunk comes first
(Algorithm 1's precedence); without the index the sets alternate; with it the
upper bursts double between lower chunks (U0 L0 U1 L1 U2 U3 L2 U4..U7 L3 ...)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include "rsr_internal.cuh"
int main() {
    const long long cases[][2] = {{20, 5}, {3, 10}, {0, 4}, {4, 0}, {1, 1}, {300, 300}, {1000, 2}, {2, 1000}};
    for (auto &c : cases)
        for (int ov = 0; ov < 2; ++ov)
            for (int grow = 0; grow < 2; ++grow) {
                rsr::ChunkWalk w(c[0], c[1], ov != 0, grow != 0);
                printf("%lld %lld %d %d:", c[0], c[1], ov, grow);
                for (long long s = 0; s < c[0] + c[1]; ++s) {
                    bool up;
                    int64_t i;
                    w.next(&up, &i);
                    printf(" %c%lld", up ? 'U' : 'L', (long long)i);
                }
                printf("\n");
            }
    return 0;
}
'''


def _walks(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "walk.cu"
    src.write_text(SRC)
    exe = tmp_path / "walk"
    inc = ["-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2604_17066_gb300", "csrc")]
    subprocess.check_call([nvcc, "-std=c++17", *inc, str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    walks = {}
    for line in out.strip().splitlines():
        head, seq = line.split(":")
        nU, nL, ov, grow = (int(x) for x in head.split())
        walks[(nU, nL, ov, grow)] = [(t[0], int(t[1:])) for t in seq.split()]
    return walks


def test_chunk_walk_orders(tmp_path):
    walks = _walks(tmp_path)
    assert len(walks) == 32
    for (nU, nL, ov, grow), seq in walks.items():
        ups = [i for s, i in seq if s == "U"]
        lows = [i for s, i in seq if s == "L"]
        assert ups == list(range(nU)) and lows == list(range(nL)), (nU, nL, ov, grow)
        if ov:
            assert [s for s, _ in seq] == ["L"] * nL + ["U"] * nU
            continue
        if nU and nL:
            assert seq[0] == ("U", 0)
        if not grow:
            m = min(nU, nL)
            assert [s for s, _ in seq[:2 * m]] == ["U", "L"] * m
        else:
            # upper chunks visited before lower chunk b: 2^b (all of them once the upper set runs out)
            where = {i: k for k, (s, i) in enumerate(seq) if s == "L"}
            for b in range(nL):
                before = sum(1 for s, _ in seq[:where[b]] if s == "U")
                assert before == min(nU, 2 ** b), (nU, nL, b, before)
    assert [s + str(i) for s, i in walks[(20, 5, 0, 1)]][:12] == \
        ["U0", "L0", "U1", "L1", "U2", "U3", "L2", "U4", "U5", "U6", "U7", "L3"]
