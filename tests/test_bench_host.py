"""Host logic of the benchmark (no GPU): the code hash that keys the profiled traffic figure."""
import bench


def _write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_code_hash_ignores_comments_and_blank_lines(tmp_path):
    a = _write(tmp_path, "a.cu", "int f(int x)\n{\n    return x + 1;  // one more\n}\n")
    b = _write(tmp_path, "b.cu", "// a header comment\nint f(int x)\n{\n\n    return x + 1;   \n}\n")
    assert bench._code_hash([a]) == bench._code_hash([b])


def test_code_hash_sees_code_changes(tmp_path):
    a = _write(tmp_path, "a.cu", "int f(int x)\n{\n    return x + 1;\n}\n")
    b = _write(tmp_path, "b.cu", "int f(int x)\n{\n    return x + 2;\n}\n")
    c = _write(tmp_path, "c.cu", "int f(int x)\n{\n    return x+1;\n}\n")  # spacing is code too
    ha, hb, hc = (bench._code_hash([p]) for p in (a, b, c))
    assert len({ha, hb, hc}) == 3


def test_code_hash_depends_on_file_order(tmp_path):
    a = _write(tmp_path, "a.cu", "int a;\n")
    b = _write(tmp_path, "b.cu", "int b;\n")
    assert bench._code_hash([a, b]) != bench._code_hash([b, a])


def test_kernel_hash_is_well_formed():
    h = bench._kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_cpu_baseline_times_a_whole_small_waveform():
    """The oracle baseline on a tiny workload: every sample computed (no extrapolation), on the
    thread count asked for, with the result returned for the accuracy check."""
    from paper_2104_04582_gb300 import workloads as W
    w = W.tiny_inputs(5, K=6, n_samples=300)
    cb, h = bench.cpu_baseline(w, target_s=0.5, threads=1, what="a tiny waveform")
    assert cb["cores"] == 1 and cb["kind"] == "oracle" and cb["unit"] == bench.UNIT
    assert cb["sample"].startswith("all 300 samples of a tiny waveform")
    assert cb["seconds_full_waveform"] == cb["seconds"] and cb["value"] > 0
    assert len(h) == 300
