"""bench.py's host-side helpers: the kernel-code hash that decides whether the
committed ncu traffic still applies, and the traffic scaling."""
import bench


SRC = """// a comment
__device__ int f(int a) {  /* block
   comment */ return a + 1;   // trailing
}
"""


def test_code_hash_ignores_comments_and_layout_but_not_code():
    def h(src, k=0):  # the source in slot k of the hashed files
        texts = [""] * len(bench.KERNEL_SOURCES)
        texts[k] = src
        return bench.kernel_source_hash(texts)

    for k in range(len(bench.KERNEL_SOURCES)):
        base = h(SRC, k)
        assert h(SRC.replace("// a comment", "// another comment"), k) == base
        assert h(SRC.replace("\n", "\n\n"), k) == base
        assert h(SRC.replace("a + 1", "a + 2"), k) != base
    assert h(SRC, 0) != h(SRC, 1)  # which file holds the code counts


def test_traffic_scales_with_cells_and_is_near_the_algorithmic_bytes():
    t = bench.measured_traffic("f32", 4194304)
    if t is None:  # the kernel changed since the committed capture: nothing to scale
        return
    # one captured launch: reads above the algorithmic half (ghost blocks), writes
    # below it (the tail of the writes is still in L2 when the launch ends)
    assert 0.8 * 152 * 4194304 < t < 1.2 * 152 * 4194304
    assert bench.measured_traffic("f32", 2 * 4194304) == 2 * t
