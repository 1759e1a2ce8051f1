"""Checkpoint and resume of the training loop (host logic, no GPU): a trainer restored from a
checkpoint holds the same parameters, Adam state, random-vector generator state and step,
so it continues bit for bit like the run that wrote it; a checkpoint of another training
setup is refused.  The optimizer steps here use fixed gradients in place of the library's
loss, which needs a GPU."""
import pytest
import torch

from paper_2102_12071_gb300 import train as T


def _trainer(seed=0, **kw):
    args = dict(sizes=(15,), per_size=2, nvec=2, lr=1e-2, seed=seed, device="cpu", net_arch="conv_shared")
    args.update(kw)
    return T.Trainer(**args)


def _fake_step(tr, g):
    """One Adam step with gradient g, plus the random vectors a real step would draw."""
    tr.opt.zero_grad(set_to_none=True)
    tr.params.grad = g.clone()
    tr.opt.step()
    z = torch.randn((tr.per_size, tr.nvec, 15, 15), generator=tr.gen, device=tr.device)
    tr.step_count += 1
    return z


def test_resume_continues_bit_for_bit(tmp_path):
    gen = torch.Generator().manual_seed(5)
    grads = [torch.randn(T.NPARAMS_SHARED, generator=gen) for _ in range(6)]
    a = _trainer()
    for g in grads[:3]:
        _fake_step(a, g)
    path = str(tmp_path / "state.pt")
    a.save_checkpoint(path)
    b = _trainer(seed=9)  # other starting parameters and generator: all overwritten
    b.load_checkpoint(path)
    assert b.step_count == a.step_count == 3
    assert torch.equal(b.params, a.params)
    sa, sb = a.opt.state_dict(), b.opt.state_dict()
    for k in ("exp_avg", "exp_avg_sq"):
        assert torch.equal(sa["state"][0][k], sb["state"][0][k])
    for g in grads[3:]:
        assert torch.equal(_fake_step(a, g), _fake_step(b, g))  # the same random vectors
        assert torch.equal(a.params, b.params)  # and the same Adam steps


def test_checkpoint_of_another_setup_is_refused(tmp_path):
    a = _trainer()
    path = str(tmp_path / "state.pt")
    a.save_checkpoint(path)
    for kw in ({"net_arch": "conv"}, {"sizes": (31,)}, {"nvec": 3}, {"max_cycles": 2}):
        with pytest.raises(ValueError):
            _trainer(**kw).load_checkpoint(path)


def test_checkpoint_write_replaces_the_file_atomically(tmp_path):
    a = _trainer()
    path = str(tmp_path / "sub" / "state.pt")
    a.save_checkpoint(path)
    _fake_step(a, torch.ones(T.NPARAMS_SHARED))
    a.save_checkpoint(path)
    assert sorted(p.name for p in (tmp_path / "sub").iterdir()) == ["state.pt"]
    b = _trainer()
    b.load_checkpoint(path)
    assert b.step_count == 1 and torch.equal(b.params, a.params)
