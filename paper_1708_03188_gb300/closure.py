"""Learned closure for an under-resolved coarse Ginzburg-Landau step (no counterpart in the paper).

A coarse step S_c (the library's Ginzburg-Landau stepper on a coarse M_c x M_c grid) is
corrected by a small periodic CNN C acting on the physical field:
    u_{n+1} = S_c(u_n) + C(u_n),
with C = conv3x3(2->32) ReLU conv3x3(32->32) ReLU conv3x3(32->32) ReLU conv3x3(32->2) (19,682
parameters), channels (Re u, Im u): BF16 weights and hidden activations, FP32 accumulation, and the
FP32 field as the first layer's input (a BF16 rounding of the field, 2^-8 relative, would be
larger than the corrections the network has to learn).  The
training targets come from fine-grid runs of the same method: a fine M_f x M_f trajectory is
spectrally truncated to the coarse wavenumbers every coarse time step, and the target is the
difference between the truncated fine state and the coarse step of the previous truncated state.
The network's forward and backward passes, the loss gradient, the optimiser update, the
spectral truncation and the field/channel conversions run in libsgm's kernels (sgm_conv3x3_*,
sgm_mse_grad, sgm_adamw_step, sgm_spectral_truncate, sgm_pack_channels, sgm_unpack_add), the
steps and transforms in its Ginzburg-Landau and space kernels; batching, target scaling and
the error norms of the evaluation use torch tensor operations.
"""
import math

import numpy as np
import torch

from . import inputs, sgm

LAYERS = [(32, 2), (32, 32), (32, 32), (2, 32)]   # (Cout, Cin)
DOMAIN = [(-50.0, 50.0), (-50.0, 50.0)]


class ClosureNet:
    def __init__(self, seed=0):
        sizes = []
        for o, c in LAYERS:
            sizes += [o * c * 9, o]
        total = sum(sizes)
        dev = "cuda"
        self.w = torch.zeros(total, dtype=torch.float32, device=dev)       # FP32 master weights
        self.wb = torch.zeros(total, dtype=torch.bfloat16, device=dev)     # BF16 copy used by the kernels
        self.g = torch.zeros_like(self.w)
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.W, self.B, self.Wb, self.gW, self.gB = [], [], [], [], []
        off = 0
        gen = torch.Generator().manual_seed(inputs.SEED_BASE + 4000 + seed)
        for li, (o, c) in enumerate(LAYERS):
            n = o * c * 9
            self.W.append(self.w[off:off + n].view(o, c, 3, 3))
            self.Wb.append(self.wb[off:off + n].view(o, c, 3, 3))
            self.gW.append(self.g[off:off + n].view(o, c, 3, 3))
            std = math.sqrt(2.0 / (c * 9)) * (0.1 if li == len(LAYERS) - 1 else 1.0)
            self.W[-1].copy_(torch.randn(o, c, 3, 3, generator=gen) * std)
            off += n
            self.B.append(self.w[off:off + o])
            self.gB.append(self.g[off:off + o])
            off += o
        self.wb.copy_(self.w.to(torch.bfloat16))
        self.steps = 0
        self.acts = None

    @property
    def num_params(self):
        return self.w.numel()

    def forward(self, x):
        """x: [B, 2, H, W] FP32 field channels -> correction [B, 2, H, W] FP32 (activations kept
        for backward)."""
        Bn, _, H, Wd = x.shape
        acts = [x]
        h = x
        for li in range(3):
            y = torch.empty((Bn, 32, H, Wd), dtype=torch.bfloat16, device=x.device)
            sgm.conv3x3_forward(h, self.Wb[li], self.B[li], y, relu=True)
            acts.append(y)
            h = y
        out = torch.empty((Bn, 2, H, Wd), dtype=torch.float32, device=x.device)
        sgm.conv3x3_forward(h, self.Wb[3], self.B[3], out, relu=False)
        self.acts = acts
        return out

    def backward(self, gout):
        """Gradients of sum(gout * forward(x)) into self.g (overwritten)."""
        self.g.zero_()
        g = gout
        for li in range(3, -1, -1):
            x_in = self.acts[li]
            sgm.conv3x3_backward_weights(g, x_in, self.gW[li], self.gB[li])
            if li > 0:
                gx = torch.empty(x_in.shape, dtype=torch.float32, device=x_in.device)
                sgm.conv3x3_backward_data(g, self.Wb[li], x_in, gx)   # x_in is a ReLU output: its mask
                g = gx

    def adam(self, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-5):
        self.steps += 1
        sgm.adamw_step(self.w, self.wb, self.g, self.m, self.v, lr, beta1, beta2, eps, weight_decay, self.steps)


class CoarseModel:
    """Ginzburg-Landau stepper (integrating-factor RK4; complex64, or complex128 with
    precision="f64") and its transforms."""

    def __init__(self, M, dt, beta=1.5, gamma=-0.5, precision="f32"):
        self.M = M
        self.dt = dt
        self.space = sgm.Space(["c2c", "c2c"], (M, M), domain=DOMAIN, precision=precision)
        self.gl = sgm.GinzburgLandau(self.space, beta, gamma, dt, "ifrk4")

    def step_batch(self, uh):
        """uh [B, M, M] complex64 spectral states; returns S_c(uh) (new tensor)."""
        out = uh.clone()
        for b in range(out.shape[0]):
            self.gl.step(out[b], 1)
        return out

    def to_physical(self, uh):
        return torch.stack([self.space.backward(uh[b]) for b in range(uh.shape[0])])

    def to_spectral(self, u):
        return torch.stack([self.space.forward(u[b]) for b in range(u.shape[0])])


def fine_trajectories(Mf, Mc, ntraj, t_spin, nsnap, dt_f, dt_c, first_item=0, beta=1.5, gamma=-0.5):
    """Truncated fine-grid states [ntraj, nsnap + 1, Mc, Mc] (complex64, spectral), sampled every
    dt_c after a spin-up of t_spin from u0 = 0.01 (N(0,1) + i N(0,1)); fine stepper: complex64
    integrating-factor RK4 with dt_f."""
    sp = sgm.Space(["c2c", "c2c"], (Mf, Mf), domain=DOMAIN, precision="f32")
    gl = sgm.GinzburgLandau(sp, beta, gamma, dt_f, "ifrk4")
    per = int(round(dt_c / dt_f))
    snaps = torch.empty((ntraj, nsnap + 1, Mc, Mc), dtype=torch.complex64, device="cuda")
    for t in range(ntraj):
        u0 = torch.from_numpy(inputs.gl_initial(Mf, first_item + t)).to(torch.complex64).cuda()
        uh = sp.forward(u0)
        gl.step(uh, int(round(t_spin / dt_f)))
        for s in range(nsnap + 1):
            sgm.spectral_truncate(uh.unsqueeze(0), snaps[t, s].unsqueeze(0))
            if s < nsnap:
                gl.step(uh, per)
    return snaps


def training_pairs(coarse, snaps):
    """(x, target): x = physical truncated state at t_n, target = truncated state at t_{n+1}
    minus the coarse step of the truncated state at t_n (both physical, complex64)."""
    cur = snaps[:, :-1].reshape(-1, coarse.M, coarse.M)
    nxt = snaps[:, 1:].reshape(-1, coarse.M, coarse.M)
    stepped = coarse.step_batch(cur)
    x = coarse.to_physical(cur)
    target = coarse.to_physical(nxt) - coarse.to_physical(stepped)
    return x, target


def as_channels(u, scale):
    """complex64 [B, M, M] -> FP32 [B, 2, M, M] channels (Re, Im) times scale."""
    return torch.stack([u.real, u.imag], dim=1).float() * scale


def as_fp32_channels(u, scale):
    return as_channels(u, scale)


def augment(u, d, gen):
    """The same random symmetry of the Ginzburg-Landau equation applied to states u and their
    corrections d ([B, M, M] complex64): a global phase exp(i theta) (U(1) invariance), a
    periodic translation, a transposition and reflections of the square grid."""
    Bn, M = u.shape[0], u.shape[1]
    theta = torch.rand(Bn, generator=gen) * (2 * math.pi)
    ph = torch.polar(torch.ones(Bn), theta).to(torch.complex64).to(u.device).view(Bn, 1, 1)
    u, d = u * ph, d * ph
    sx, sy = (int(v) for v in torch.randint(0, M, (2,), generator=gen))
    u, d = torch.roll(u, (sx, sy), (1, 2)), torch.roll(d, (sx, sy), (1, 2))
    if bool(torch.randint(0, 2, (1,), generator=gen)):
        u, d = u.transpose(1, 2), d.transpose(1, 2)
    for ax in (1, 2):
        if bool(torch.randint(0, 2, (1,), generator=gen)):
            # x -> -x on the periodic mesh x_j = -L/2 + L j / M maps index j to (M - j) mod M
            idx = (-torch.arange(M, device=u.device)) % M
            u, d = u.index_select(ax, idx), d.index_select(ax, idx)
    return u.contiguous(), d.contiguous()


def train(net, x, target, iters=400, batch=16, lr=2e-3, seed=0, log=None, symmetries=True):
    """Minimise the MSE between net(x) and the scaled target with AdamW and a cosine learning-
    rate decay, each minibatch transformed by a random symmetry of the equation (the transform of
    augment, done on the device by sgm.augment_pack); returns the loss history and the target
    scale (the network predicts target / scale).

    Every minibatch's pool indices, phases, translation and reflections are drawn up front from
    the host generator and uploaded once, so an iteration is device work only: one transform
    launch, the network's kernels and the AdamW step."""
    scale_t = 1.0 / max(float(target.abs().pow(2).mean().sqrt()), 1e-30)
    n, M = x.shape[0], x.shape[-1]
    nb = min(batch, n)
    gen = torch.Generator(device="cpu").manual_seed(inputs.SEED_BASE + 4100 + seed)
    idx_all = torch.randint(0, n, (iters, nb), generator=gen).to(torch.int32)
    if symmetries:
        theta = torch.rand(iters, nb, generator=gen, dtype=torch.float64) * (2 * math.pi)
        shift = torch.randint(0, M, (iters, 2), generator=gen).tolist()
        bits = torch.randint(0, 2, (iters, 3), generator=gen).tolist()
        flags = [t * sgm.AUG_TRANSPOSE + f0 * sgm.AUG_FLIP0 + f1 * sgm.AUG_FLIP1 for t, f0, f1 in bits]
    else:
        theta = torch.zeros(iters, nb, dtype=torch.float64)
        shift = [[0, 0]] * iters
        flags = [0] * iters
    idx_all = idx_all.cuda()
    ph_all = torch.polar(torch.ones_like(theta), theta).to(torch.complex64).cuda()
    xs, ts = x.contiguous(), target.contiguous()
    xb = torch.empty((nb, 2, M, M), dtype=torch.float32, device="cuda")
    tb = torch.empty_like(xb)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for it in range(iters):
        sgm.augment_pack(xs, ts, idx_all[it], ph_all[it], shift[it][0], shift[it][1], flags[it], 1.0, scale_t,
                         xb, tb)
        out = net.forward(xb)
        gout = torch.empty_like(out)
        loss.zero_()
        sgm.mse_grad(out, tb, gout, loss)
        net.backward(gout)
        net.adam(lr=lr * 0.5 * (1.0 + math.cos(math.pi * it / iters)))
        if it % 50 == 0 or it == iters - 1:
            hist.append(float(loss.item()))
            if log:
                log(it, hist[-1])
    return hist, scale_t


def corrected_step(coarse, net, uh, scale_t):
    """S_c(uh) + C(uh) for a batch of spectral states (returns spectral states)."""
    u_phys = coarse.to_physical(uh)
    corr = net.forward(as_channels(u_phys, 1.0))
    stepped = coarse.to_physical(coarse.step_batch(uh))
    sgm.unpack_add(corr, stepped, 1.0 / scale_t)
    return coarse.to_spectral(stepped)


def relative_errors(coarse, net, snaps, scale_t, horizon=1):
    """Mean relative L2 error after `horizon` coarse steps against the truncated fine states, for
    the plain coarse step and the corrected one."""
    start = snaps[:, :-horizon].reshape(-1, coarse.M, coarse.M)
    truth = snaps[:, horizon:].reshape(-1, coarse.M, coarse.M)
    plain, learned = start.clone(), start.clone()
    for _ in range(horizon):
        plain = coarse.step_batch(plain)
        learned = corrected_step(coarse, net, learned, scale_t)
    tn = torch.linalg.vector_norm(truth.reshape(truth.shape[0], -1), dim=1)
    ep = torch.linalg.vector_norm((plain - truth).reshape(truth.shape[0], -1), dim=1) / tn
    el = torch.linalg.vector_norm((learned - truth).reshape(truth.shape[0], -1), dim=1) / tn
    return float(ep.mean()), float(el.mean())


def graphed(fn):
    """Capture fn() - device work on the current stream into buffers that stay fixed - into a
    CUDA graph after one eager warm-up run; returns a function that replays the graph."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g.replay



def _energy_and_spectrum(uh, kbins):
    """<|u|^2> (Parseval: the sum of |u_hat|^2 with the transform's 1/M^2) and the radial energy
    spectrum (sum of |u_hat|^2 over the integer shells |k| in [s, s + 1)) of spectral states."""
    e = uh.abs().pow(2)
    energy = e.sum(dim=(1, 2))
    spec = torch.zeros((uh.shape[0], int(kbins.max()) + 1), device=uh.device)
    spec.index_add_(1, kbins.reshape(-1), e.reshape(uh.shape[0], -1).float())
    return energy, spec


def long_horizon(coarse, net, scale_t, Mf=256, nstates=4, nsteps=2000, t_spin=30.0, dt_f=0.01, first_item=200,
                 beta=1.5, gamma=-0.5):
    """Statistics over a long horizon (nsteps coarse steps of coarse.gl's dt) from held-out states:
    the fine run (complex64 IF-RK4 on Mf^2 with dt_f), spectrally truncated to the coarse grid every
    coarse step, against the plain coarse run and the corrected one.  The flow is chaotic, so the
    trajectories decorrelate; what a closure can get right is the statistics.  Returns the relative
    errors of the time-averaged <|u|^2> and of the time-averaged radial energy spectrum over the
    second half of the horizon, for the plain and the learned coarse runs."""
    Mc = coarse.M
    dt_c = coarse.dt
    sp = sgm.Space(["c2c", "c2c"], (Mf, Mf), domain=DOMAIN, precision="f32")
    gl = sgm.GinzburgLandau(sp, beta, gamma, dt_f, "ifrk4")
    per = int(round(dt_c / dt_f))
    fine = [sp.forward(torch.from_numpy(inputs.gl_initial(Mf, first_item + s)).to(torch.complex64).cuda())
            for s in range(nstates)]
    for uh in fine:
        gl.step(uh, int(round(t_spin / dt_f)))
    start = torch.empty((nstates, Mc, Mc), dtype=torch.complex64, device="cuda")
    for s, uh in enumerate(fine):
        sgm.spectral_truncate(uh.unsqueeze(0), start[s].unsqueeze(0))
    l = torch.from_numpy(np.fft.fftfreq(Mc, 1.0 / Mc)).cuda()
    kbins = torch.sqrt(l[:, None] ** 2 + l[None, :] ** 2).floor().long()
    plain, learned = start.clone(), start.clone()
    acc = {name: [0.0, 0.0] for name in ("fine", "plain", "learned")}
    trunc = torch.empty_like(start)
    half = nsteps // 2
    for n in range(1, nsteps + 1):
        for s, uh in enumerate(fine):
            gl.step(uh, per)
            sgm.spectral_truncate(uh.unsqueeze(0), trunc[s].unsqueeze(0))
        plain = coarse.step_batch(plain)
        learned = corrected_step(coarse, net, learned, scale_t)
        if n > half:
            for name, st in (("fine", trunc), ("plain", plain), ("learned", learned)):
                e, spec = _energy_and_spectrum(st, kbins)
                acc[name][0] = acc[name][0] + e.mean()
                acc[name][1] = acc[name][1] + spec.mean(dim=0)
    gl.close()
    sp.close()
    ef, sf = acc["fine"]
    out = {"horizon_steps": nsteps, "time_units": round(nsteps * dt_c, 3), "states": nstates,
           "averaged_over": "second half of the horizon"}
    for name in ("plain", "learned"):
        e, spec = acc[name]
        out[name] = {"energy_rel_error": float(abs(e - ef) / ef),
                     "spectrum_rel_l2": float(torch.linalg.vector_norm(spec - sf) / torch.linalg.vector_norm(sf)),
                     "finite": bool(torch.isfinite(e).item())}
    out["fine_energy"] = float(ef / (nsteps - half))
    return out
