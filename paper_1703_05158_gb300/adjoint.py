"""torch.autograd.Function over the differentiation form: the mean plate
drag J(theta) of a Channel, theta = (inlet peak velocity, body force, Cs),
with its gradient from the library's hand-written adjoint
(lbm_channel_backward; checkpoint and recompute inside the library)."""
import torch


class ChannelDrag(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, channel):
        th = tuple(float(v) for v in theta.detach().to("cpu", torch.float64))
        channel.set_theta(th)
        J = channel.forward()
        ctx.channel, ctx.theta = channel, th
        return theta.new_tensor(J)

    @staticmethod
    def backward(ctx, gJ):
        ch = ctx.channel
        if ch.theta != ctx.theta:  # another forward ran in between: its checkpoints are not ours
            ch.set_theta(ctx.theta)
            ch.forward()
        g = torch.as_tensor(ch.backward(), dtype=gJ.dtype, device=gJ.device)
        return gJ * g, None


def plate_drag(theta, channel):
    """J(theta) as a differentiable tensor (theta: 3 values)."""
    return ChannelDrag.apply(theta, channel)
