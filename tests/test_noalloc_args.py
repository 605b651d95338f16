"""Argument checks of the allocation-free conversion's Python binding (CPU).

mhdc_build_noalloc writes into arrays the caller owns and passes the C layer
raw pointers, so a host tensor, a short tensor or a tensor of the wrong type
would be written out of bounds by the conversion kernels.  The binding checks
every argument before anything runs on the GPU; these tests drive those
checks with stand-in tensors (no GPU needed) and expect each wrong argument
to raise.
"""
import pytest

torch = pytest.importorskip("torch")
import paper_2105_04937_gb300 as mh  # noqa: E402


class Fake:
    """The attributes of a torch tensor the checks read."""

    def __init__(self, dtype, numel, device="cuda:0", contiguous=True):
        self.dtype = dtype
        self._n = numel
        self.device = torch.device(device)
        self.is_cuda = self.device.type == "cuda"
        self._c = contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


N, NNZ, NB, CAP_P = 1000, 5000, 64, 40


def good(dtype="f64"):
    vt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    nb = (N + NB - 1) // NB
    return dict(row_ptr=Fake(torch.int32, N + 1), col=Fake(torch.int32, NNZ),
                val=Fake(torch.float64, NNZ), dia_ptr=Fake(torch.int32, nb + 1),
                dia_offset=Fake(torch.int32, CAP_P), dia_val=Fake(vt, CAP_P * NB),
                csr_row_ptr=Fake(torch.int32, N + 1), csr_col=Fake(torch.int32, NNZ),
                csr_val=Fake(vt, NNZ))


def run(a, dtype="f64", n=N, nnz=NNZ, n_b=NB):
    return mh._noalloc_check(n, nnz, a["row_ptr"], a["col"], a["val"], n_b, mh.DTYPES[dtype],
                             a["dia_ptr"], a["dia_offset"], a["dia_val"], a["csr_row_ptr"],
                             a["csr_col"], a["csr_val"])


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_valid_arguments_pass(dtype):
    assert run(good(dtype), dtype) == (CAP_P, NNZ)


def test_bf16_values_may_be_int16_bits():
    a = good("bf16")
    a["dia_val"] = Fake(torch.int16, CAP_P * NB)
    a["csr_val"] = Fake(torch.int16, NNZ)
    assert run(a, "bf16") == (CAP_P, NNZ)


INT_ARRAYS = ["row_ptr", "col", "dia_ptr", "dia_offset", "csr_row_ptr", "csr_col"]
SIZED = {"row_ptr": N + 1, "col": NNZ, "val": NNZ, "dia_ptr": (N + NB - 1) // NB + 1,
         "csr_row_ptr": N + 1, "dia_val": CAP_P * NB}


@pytest.mark.parametrize("name", list(good()))
def test_host_tensor_is_rejected(name):
    a = good()
    f = a[name]
    a[name] = Fake(f.dtype, f.numel(), device="cpu")
    with pytest.raises(ValueError, match="CUDA"):
        run(a)


@pytest.mark.parametrize("name", list(good()))
def test_other_device_is_rejected(name):
    a = good()
    f = a[name]
    a[name] = Fake(f.dtype, f.numel(), device="cuda:1")
    if name == "row_ptr":
        a = {k: (Fake(v.dtype, v.numel(), device="cuda:0") if k == "row_ptr" else
                 Fake(v.dtype, v.numel(), device="cuda:1")) for k, v in a.items()}
    with pytest.raises(ValueError, match="is on"):
        run(a)


@pytest.mark.parametrize("name", list(good()))
def test_non_contiguous_is_rejected(name):
    a = good()
    f = a[name]
    a[name] = Fake(f.dtype, f.numel(), contiguous=False)
    with pytest.raises(ValueError, match="contiguous"):
        run(a)


@pytest.mark.parametrize("name", INT_ARRAYS)
def test_index_arrays_must_be_int32(name):
    a = good()
    a[name] = Fake(torch.int64, a[name].numel())
    with pytest.raises(TypeError):
        run(a)


@pytest.mark.parametrize("name,dtype,bad", [
    ("val", "f64", torch.float32), ("dia_val", "f64", torch.float32),
    ("csr_val", "f64", torch.int64), ("dia_val", "f32", torch.float64),
    ("csr_val", "f32", torch.bfloat16), ("dia_val", "bf16", torch.float32),
    ("csr_val", "bf16", torch.float16)])
def test_value_arrays_must_match_the_storage_type(name, dtype, bad):
    a = good(dtype)
    a[name] = Fake(bad, a[name].numel())
    with pytest.raises(TypeError):
        run(a, dtype)


@pytest.mark.parametrize("name", list(SIZED))
def test_short_arrays_are_rejected(name):
    a = good()
    a[name] = Fake(a[name].dtype, SIZED[name] - 1)
    with pytest.raises(ValueError):
        run(a)


def test_bad_sizes_are_rejected():
    with pytest.raises(ValueError):
        run(good(), n=0)
    with pytest.raises(ValueError):
        run(good(), n_b=0)
    with pytest.raises(ValueError):
        run(good(), nnz=-1)
