"""The key under which bench.py keeps the committed DRAM traffic: the stage kernels' code with its
comments removed, so that a comment edit keeps the traffic and a code edit drops it."""
import bench


def test_strip_comments_keeps_code_and_literals():
    src = 'int a = 1; // note\n/* block\n   comment */ const char* s = "// not a comment";\n\n  char q = \'"\';  \n'
    assert bench.strip_comments(src) == 'int a = 1;\n  const char* s = "// not a comment";\n  char q = \'"\';'


def test_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2311_04989_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.STAGE_SOURCES:
        (csrc / f).write_text("__global__ void k(float* x) { x[0] = 1.f; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "mlp.cuh").write_text("// a new comment\n__global__ void k(float* x) { x[0] = 1.f; }  /* c */\n")
    assert bench.kernel_source_hash() == h0
    (csrc / "mlp.cuh").write_text("__global__ void k(float* x) { x[0] = 2.f; }\n")
    assert bench.kernel_source_hash() != h0
