"""GPU FNO training kernels and the differentiable hybrid step against FP64 references.

  * fno_train_forward against the numpy FNO oracle (Sec. 2.2);
  * fno_train_backward (the spectral layer's adjoint, 1x1 layers, activations, lifting
    and decoder) against torch autograd through oracle/grad_oracle.py's FP64 FNO;
  * the whole training objective -- FNO prediction, re-initialisation, LBM steps, MSE
    of (rho, u) -- differentiated through both adjoints, against the FP64 reference.
FP32 parameters that are exactly representable in bfloat16 are used, so that the
oracle (which rounds parameters to bfloat16) and the FP32 training path see the same
values.  Bar: 1e-4 relative L2 per gradient tensor (FP32 against FP64).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import fno_oracle as fo
from oracle import grad_oracle as go

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300.fno import FnoShape  # noqa: E402
from paper_2604_27158_gb300.lbm import GridSpec, Lattice  # noqa: E402
from paper_2604_27158_gb300.train import fno_apply, fno_train_query, hybrid_loss  # noqa: E402

REL = 1e-4


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shapes(width, layers, modes, dec_size, act=0, dec_layers=1):
    s = synth.FnoShape(width=width, layers=layers, modes=modes, dec_size=dec_size,
                       dec_layers=dec_layers)
    g = FnoShape(width=width, layers=layers, modes=modes, dec_size=dec_size,
                 dec_layers=dec_layers, activation=act)
    return s, g


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


CASES = [(8, 2, 3, 8, 0, 1, 2, 16, 24), (32, 2, 6, 32, 0, 1, 2, 32, 64),
         (16, 1, 4, 12, 1, 2, 1, 20, 40)]


@pytest.mark.parametrize("width,layers,modes,dec,act,dec_layers,B,H,W", CASES)
def test_training_forward_and_backward_match_fp64(width, layers, modes, dec, act, dec_layers,
                                                  B, H, W):
    _requires_gpu()
    s, g = _shapes(width, layers, modes, dec, act, dec_layers)
    params = synth.fno_random_params(s, seed=3, out_scale=1.0)
    flat = synth.fno_flatten_params(s, params).astype(np.float32)
    assert fno_train_query(g, B, H, W).n_params == flat.size
    rng = np.random.default_rng(7)
    x = fo.bf16(rng.standard_normal((B, 4, H, W))).astype(np.float32)
    dout = rng.standard_normal((B, 3, H, W)).astype(np.float32)
    pt = torch.from_numpy(flat).cuda().requires_grad_(True)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    y = fno_apply(g, pt, xt)
    (y * torch.from_numpy(dout).cuda()).sum().backward()
    act_name = "gelu" if act == 0 else "relu"
    ref = fo.fno_forward(s, params, x, activation=act_name)
    e = _rel(y.detach().cpu().numpy(), ref)
    print(f"train forward C={width} L={layers} m={modes}: rel L2 {e:.2e}")
    assert e < REL
    # FP64 reference gradients
    P64 = go.bf16_params(params, requires_grad=True)
    x64 = torch.from_numpy(x.astype(np.float64)).requires_grad_(True)
    y64 = go.fno_forward(s, P64, x64, activation=act_name)
    (y64 * torch.from_numpy(dout.astype(np.float64))).sum().backward()
    got = pt.grad.detach().cpu().numpy()
    off = 0
    for name, shp in synth.fno_param_shapes(s):
        n = int(np.prod(shp))
        e = _rel(got[off:off + n], P64[name].grad.numpy().ravel())
        print(f"  d{name}: rel L2 {e:.2e}")
        assert e < REL, name
        off += n
    e = _rel(xt.grad.detach().cpu().numpy(), x64.grad.numpy())
    print(f"  dx: rel L2 {e:.2e}")
    assert e < REL


def test_hybrid_training_gradient_matches_fp64():
    """B = 2 porous grids 32 x 32, FNO (C = 8, 2 layers, m = 4) on (rho-1, u, mask) of the
    rest state, 8 LBM steps (checkpoints every 3), loss = MSE of (rho, u) over fluid cells
    of the whole batch."""
    _requires_gpu()
    s, g = _shapes(8, 2, 4, 8)
    params = synth.fno_random_params(s, seed=11, out_scale=1e-1)
    flat = synth.fno_flatten_params(s, params).astype(np.float32)
    grids, masks = [], []
    for k in range(2):
        solid, _, _ = synth.porous_media(32, 32, 3, 4, seed=30 + k)
        grids.append(GridSpec(32, 32, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                              west_value=1.01, east_value=1.0))
        masks.append(solid)
    lat = Lattice(grids, masks)
    x = np.stack([np.stack([np.zeros((32, 32)), np.zeros((32, 32)), np.zeros((32, 32)),
                            m.astype(np.float64)]) for m in masks]).astype(np.float32)
    tg = [synth.smooth_macro_fields(32, 32, seed=50 + k, drho=1e-2, umax=0.02) for k in range(2)]
    target = [torch.from_numpy(np.concatenate([t[c].ravel() for t in tg])).cuda() for c in range(3)]
    pt = torch.from_numpy(flat).cuda().requires_grad_(True)
    loss = hybrid_loss(lat, g, pt, torch.from_numpy(x).cuda(), 8, target, every=3)
    loss.backward()
    got = pt.grad.detach().cpu().numpy()
    # FP64 reference: the batch loss is the fluid-count-weighted sum of per-grid losses
    nfl = [int((~m).sum()) for m in masks]
    P64 = go.bf16_params(params, requires_grad=True)
    total = 0.0
    for k in range(2):
        og = oracle.Grid(nx=32, ny=32, tau=0.7, bc_west=1, bc_east=1, west_value=1.01,
                         east_value=1.0)
        tl = go.TorchLattice(og, masks[k])
        tgt = tuple(torch.from_numpy(np.asarray(tg[k][c], np.float64)) for c in range(3))
        lk = go.hybrid_loss(tl, s, P64, torch.from_numpy(x[k:k + 1].astype(np.float64)), 8, tgt)
        total = total + lk * (nfl[k] / sum(nfl))
    total.backward()
    print(f"hybrid loss gpu {float(loss):.6e} fp64 {float(total):.6e}")
    assert abs(float(loss) - float(total)) <= 1e-5 * abs(float(total))
    off = 0
    for name, shp in synth.fno_param_shapes(s):
        n = int(np.prod(shp))
        e = _rel(got[off:off + n], P64[name].grad.numpy().ravel())
        print(f"  d{name}: rel L2 {e:.2e}")
        assert e < REL, name
        off += n
    lat.close()


def test_a_few_optimiser_steps_reduce_the_loss():
    """Sanity of the assembled training step: Adam on the hybrid objective lowers it."""
    _requires_gpu()
    s, g = _shapes(8, 1, 4, 8)
    params = synth.fno_random_params(s, seed=2, out_scale=1e-1)
    pt = torch.nn.Parameter(torch.from_numpy(synth.fno_flatten_params(s, params)
                                             .astype(np.float32)).cuda())
    solid, _, _ = synth.porous_media(64, 32, 3, 4, seed=4)
    lat = Lattice([GridSpec(64, 32, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                            west_value=1.01, east_value=1.0)], [solid])
    x = torch.from_numpy(np.stack([np.zeros((32, 64)), np.zeros((32, 64)), np.zeros((32, 64)),
                                   solid.astype(np.float64)])[None].astype(np.float32)).cuda()
    t = synth.smooth_macro_fields(64, 32, seed=9, drho=1e-3, umax=0.01)
    target = [torch.from_numpy(np.asarray(a).ravel()).cuda() for a in t]
    opt = torch.optim.Adam([pt], lr=1e-3)
    losses = []
    for _ in range(15):
        opt.zero_grad()
        loss = hybrid_loss(lat, g, pt, x, 8, target, every=4)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    print("losses", [f"{v:.3e}" for v in losses])
    assert losses[-1] < 0.5 * losses[0]
    lat.close()


def test_supervised_steady_training_lowers_the_prediction_error():
    """The steady framework's offline training (Sec. 2.3) with the library's kernels: LBM
    steady states of small porous media, a few hundred Adam steps; the trained parameters
    (normalisation folded into the output layer) predict the held-out states better than
    the initial ones through the inference path."""
    _requires_gpu()
    from paper_2604_27158_gb300 import steady_training as stt
    from paper_2604_27158_gb300.fno import Fno
    g = GridSpec(128, 64, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                 west_value=1.001, east_value=1.0)
    masks = [synth.porous_media(128, 64, 3, 6, seed=700 + k)[0] for k in range(20)]
    y = stt.steady_states(g, masks, 3000)
    x = stt.fno_inputs(masks)
    fl = ~torch.from_numpy(np.stack(masks)).cuda()
    s, shape = _shapes(16, 2, 6, 16)
    p0 = synth.fno_flatten_params(s, synth.fno_random_params(s, seed=3, out_scale=1.0))
    p1, hist = stt.train_supervised(shape, p0, x[:16], y[:16], fl[:16], 300, batch=4, lr=2e-3,
                                    log_every=50)
    print("loss", [f"{v:.3e}" for v in hist])

    def heldout(params):
        net = Fno(shape, params)
        pred = torch.empty_like(y[16:])
        net(x[16:], pred)
        e = float((pred - y[16:]).permute(1, 0, 2, 3)[:, fl[16:]].norm() /
                  y[16:].permute(1, 0, 2, 3)[:, fl[16:]].norm())
        net.close()
        return e

    e0, e1 = heldout(p0), heldout(p1)
    print(f"held-out rel L2: initial {e0:.3e}, trained {e1:.3e}")
    assert hist[-1] < 0.5 * hist[0]
    assert e1 < 0.5 * e0
