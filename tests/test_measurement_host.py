"""Host-side pieces of the measurement tools (no GPU): the HEALPix ring table that the
ring-FFT / cuFFT comparison groups rings by, and the keying of the committed DRAM-traffic
captures that the bench line reads."""
import numpy as np

import synthetic as S
from profile_step import ring_table


def test_ring_table_tiles_the_sphere_ring_by_ring():
    for N in (1, 2, 8, 32):
        t = ring_table(N)
        assert len(t) == 4 * N - 1
        assert t[0] == (0, 4)
        assert sum(n for _, n in t) == 12 * N * N
        assert all(t[k][0] + t[k][1] == t[k + 1][0] for k in range(len(t) - 1))
        # ring lengths 4i in the caps, 4N in the belt, mirrored north/south
        assert [n for _, n in t] == [n for _, n in reversed(t)]
        z, _ = S.pixel_positions(N)
        for first, n in t:
            assert np.ptp(z[first:first + n]) < 1e-12   # one ring = one latitude
        zr = [z[f] for f, _ in t]
        assert all(a > b for a, b in zip(zr, zr[1:]))    # north to south


def _kernel_tree(tmp_path, impl, f2):
    d = tmp_path / "paper_2606_06175_gb300" / "csrc"
    d.mkdir(parents=True, exist_ok=True)
    (d / "akra_legendre_impl.cuh").write_text(impl)
    (d / "akra_legendre_f32x2.cuh").write_text(f2)
    return str(tmp_path)


def test_kernel_source_hash_follows_code_not_comments(tmp_path, monkeypatch):
    """The key of a DRAM-traffic capture: a comment or blank-line edit keeps it, a code edit
    changes it."""
    import bench

    code = "int f(int x) {\n    return x + 1;\n}\n"
    f2 = "#define M(a) (a) /* one */ \\\n    + 1\n"
    monkeypatch.setattr(bench, "ROOT", _kernel_tree(tmp_path / "a", code, f2))
    h0 = bench.kernel_source_sha()
    monkeypatch.setattr(bench, "ROOT", _kernel_tree(
        tmp_path / "b", "// header\nint f(int x) {\n\n    return x + 1;   // add one\n}\n",
        "#define M(a) (a) /* another\n   comment */ \\\n    + 1\n"))
    assert bench.kernel_source_sha() == h0
    monkeypatch.setattr(bench, "ROOT", _kernel_tree(tmp_path / "c", code.replace("+ 1", "+ 2"), f2))
    assert bench.kernel_source_sha() != h0


def test_captured_traffic_reads_only_a_capture_of_the_current_source(tmp_path, monkeypatch):
    import bench

    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    sha = bench.kernel_source_sha()
    k = "k_leg_adjoint<float,4,1,128>"
    assert bench.captured_traffic(k)[0] is None   # no file
    (tmp_path / "legendre_traffic_des2048.md").write_text(
        "text\n"
        f"bench-traffic: kernel={k} source={sha} dram_bytes_per_launch=1234\n"
        "bench-traffic: kernel=k_leg_synth<float,1,1,128> source=000000000000 dram_bytes_per_launch=5\n")
    assert bench.captured_traffic(k)[0] == 1234.0
    b, note = bench.captured_traffic("k_leg_synth<float,1,1,128>")
    assert b is None and "older kernel source" in note
    assert bench.captured_traffic("k_leg_adjoint<float,5,1,128>")[0] is None
